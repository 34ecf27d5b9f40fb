// Partition scan for k <= 16 on the 5th-generation tensor cores: the
// screening scan of Section 3.5's search (every probed partition scored
// against the queries that probe it) with work items pipelined across each
// other and a fixed-cost screening epilogue.
//
// Work items are (partition p, up to 128 of the queries probing p), claimed
// by one persistent CTA per SM.  The item's queries are the A operand (M =
// 128 rows, K-major core-matrix layout); the partition's rows stream through
// a ring of 64-row B tiles copied by cp.async.bulk straight from the index;
// one thread issues the MMAs (kind::tf32 for fp32 rows; kind::f16 with the
// fp32 query split into bf16 hi + lo parts for bf16 rows) into one of four
// TMEM accumulators of 64 columns.
//
// Pipelining.  The producer publishes the next item's description before it
// streams the current item's tiles and never waits for an item boundary, so
// the tile ring stays full across items.  The A operand is double-buffered
// (items alternate): the epilogue loads the next item's query ids at the
// start of the current item and, after its first tile (the MMAs of the item
// before, the last readers of the other buffer, have then completed), copies
// their rows into the other buffer, which it hands to the MMA issuer two
// tiles later; the MMA issuer runs on into the next item while the epilogue
// finishes the current one.
//
// Screening (exactness as in the tensor-core scan of scan_tc.cu): a screened
// score s~ lies within delta / 2 of the fp32 dot product, delta = dscale *
// ||q|| * max_p ||x||.  The rows of a partition fall into disjoint groups of
// four; the k-th largest group maximum seen so far, a_k, is the screened
// score of k distinct rows, so the partition's k-th best exact score exceeds
// a_k - delta / 2 and a row with s~ < a_k - 2 delta cannot be in the top k.
// Per tile each epilogue thread (one query) gets the 16 group maxima from
// the TMEM load itself (tcgen05.ld.red; from an item's third tile on, a full
// tile is taken as 8 groups of eight rows, which halves the network), sorts
// them (bitonic network) and merges them into the 16 largest so far (groups
// of different sizes are still disjoint), raises its cut max(a_k - 2 delta,
// G_q - delta) (G_q: the best bound the query's finished partitions
// published), and appends the rows at or above the cut to the slot's
// candidate list in shared memory: each thread parks in shared memory only
// its groups whose maximum reaches the cut and reads them back, one loop
// trip per such group.  The cost of a tile barely depends on how
// many rows survive, so no warp waits long on its lane with the most
// survivors.  Once a slot's shared list is full its further candidates go
// straight to the pair's list in global memory; at the end of an item the
// shared entries still at or above the final cut follow, all as (s~ + delta,
// row).  The pair's header gets L_k = a_k - delta and the list length (bit
// 31: overflow of the global list, the finishing kernel then rescans the
// partition exactly); finish_queries rescores the candidates whose upper
// bound reaches the query's best L_k.
//
// Warp roles: 0 = producer (item descriptions, bulk copies), 1 = MMA issuer
// (TMEM owner), 2 = gate (does the mbarrier waits for the MMA issuer and hands
// each tile over through a named barrier), 3..6 = epilogue (query slot
// 32 * (warp % 4) + lane, its TMEM lane).  Every mbarrier wait is bounded; on
// expiry the CTA raises *err, stops, waits (bounded) for its copies and MMAs
// in flight, frees its TMEM and returns.
#include "scan_common.cuh"
#include "tc.cuh"

namespace soar {

namespace {

constexpr int kM = 128;        // query slots per item (MMA M)
constexpr int kN = 64;         // rows per tile (MMA N)
constexpr int kThreads = 224;  // producer, MMA issuer, gate, 4 epilogue warps
constexpr int kMaxStages = 8;
constexpr int kNB = 4;         // TMEM accumulators (kN columns each)
constexpr int kRing = 4;       // item descriptions in flight
constexpr int kGK = 16;        // group maxima kept per query (k <= kGK)
constexpr int kCap = 32;       // candidate rows held per query slot in shared memory
constexpr int kStageAt = 2;    // the next item's A buffer is released after this many tiles of the current one

struct GmParams {
  IvfWork work;
  const void* rows;        // index rows (fp32 or bf16), core-matrix layout, 8-row groups
  const int64_t* gstart;   // [c + 1] first 8-row group of each partition
  const float* pmax;       // [c] largest ||x|| of each partition
  const void* Qa;          // fp32 [nq][kp] query rows, or bf16 [nq][2][kp] (hi row, lo row)
  const float* qnorm;      // [nq]
  int kp;                  // K, a multiple of 8 (fp32) or 16 (bf16)
  float dscale;            // delta / (||q|| max_p ||x||)
  int k;
  int stages;
  long long wait_limit;
  int* counter;            // work-item counter
  int* err;                // set to 1 when a wait expired
  unsigned* gbound;        // [nq] ordered key of the query's best published L_k
  Cand* cand;              // [pairs][kGmList] (upper bound, row-major row position), written at an item's end
  int2* hdr;               // [pairs] (L_k as float bits, count | overflow << 31)
};

__device__ __forceinline__ unsigned ordered_key(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unordered_key(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// A work item: partition p (-1: no more items), its first pair slot and
// query count, its row count, first 8-row group and group count.
struct Item {
  int p, nqi, nrows, ng;
  int64_t e0, g0, row0;
};

__device__ Item describe(const GmParams& P, int item, int total) {
  Item d{};
  d.p = -1;
  if (item >= total) return d;
  const int oi = P.work.partition_of(item);
  const int p = P.work.order[oi];
  d.p = p;
  d.e0 = P.work.pair_off[p] + (int64_t)(item - P.work.item_base[oi]) * kM;
  d.nqi = (int)min((int64_t)kM, P.work.pair_off[p + 1] - d.e0);
  d.row0 = P.work.part_off[p];
  d.nrows = (int)(P.work.part_off[p + 1] - d.row0);
  d.g0 = P.gstart[p];
  d.ng = (int)(P.gstart[p + 1] - d.g0);
  return d;
}


// KX = 10: k fixed at 10 (the k-th of the sorted group maxima is a fixed
// register); KX = 0: k <= 16 at run time.
template <typename ET, int KX>
__global__ void __launch_bounds__(kThreads, 1) scan_gm_kernel(GmParams P) {
  constexpr uint32_t es = sizeof(ET);            // bytes per operand element
  constexpr unsigned kFull = 0xffffffffu;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int kp = P.kp, S = P.stages;
  const int k = KX > 0 ? KX : P.k;
  const uint32_t sbo = (uint32_t)kp * 8u * es;         // bytes between 8-row groups
  const uint32_t a_part = (uint32_t)kM * kp * es;      // one A part (bf16: hi or lo)
  const uint32_t a_bytes = (es == 4 ? 1u : 2u) * a_part;   // one A operand buffer
  const uint32_t b_bytes = (uint32_t)kN * kp * es;
  const char* rows = static_cast<const char*>(P.rows);
  unsigned char* sA = base;                            // two A operand buffers (items alternate)
  unsigned char* sB = base + 2 * a_bytes;
  // a tile's surviving groups parked per query slot as float4s ([group][kM],
  // so that a warp's 32 lanes write 512 consecutive bytes), then the
  // candidates per query slot ([entry][kM]: 32 lanes, 32 distinct banks):
  // scores, then padded row positions
  float4* park_s = reinterpret_cast<float4*>(sB + (size_t)S * b_bytes);
  float* list_s = reinterpret_cast<float*>(park_s + 16 * kM);
  uint64_t* bars = reinterpret_cast<uint64_t*>(list_s + 2 * kCap * kM);
  // bars: full[S], empty[S], tfull[kNB], tempty[kNB], dfull[kRing], dempty[kRing], aready[2], agone[2]
  __shared__ Item ring_s[kRing];
  __shared__ uint32_t abuf_s[2];                       // A buffer of the tile handed to the MMA issuer
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  __shared__ int issued_s, consumed_s, committed_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int s) { return tc::smem_u32(&bars[s]); };
  auto empty = [&](int s) { return tc::smem_u32(&bars[S + s]); };
  auto tfull = [&](int b) { return tc::smem_u32(&bars[2 * S + b]); };
  auto tempty = [&](int b) { return tc::smem_u32(&bars[2 * S + kNB + b]); };
  auto dfull = [&](int r) { return tc::smem_u32(&bars[2 * S + 2 * kNB + r]); };
  auto dempty = [&](int r) { return tc::smem_u32(&bars[2 * S + 2 * kNB + kRing + r]); };
  auto aready = [&](int a) { return tc::smem_u32(&bars[2 * S + 2 * kNB + 2 * kRing + a]); };
  // the gate has seen buffer a's staged item (so the epilogue never readies
  // a buffer twice before the gate has waited once)
  auto agone = [&](int a) { return tc::smem_u32(&bars[2 * S + 2 * kNB + 2 * kRing + 2 + a]); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::bar_init(full(s), 1);
      tc::bar_init(empty(s), 1);
    }
    for (int b = 0; b < kNB; ++b) {
      tc::bar_init(tfull(b), 1);
      tc::bar_init(tempty(b), 4);
    }
    for (int r = 0; r < kRing; ++r) {
      tc::bar_init(dfull(r), 1);
      tc::bar_init(dempty(r), 5);                      // the gate and the four epilogue warps
    }
    tc::bar_init(aready(0), 4);
    tc::bar_init(aready(1), 4);
    tc::bar_init(agone(0), 1);
    tc::bar_init(agone(1), 1);
    tc::bar_init_fence();
    abort_s = 0;
    issued_s = consumed_s = committed_s = 0;
  }
  if (warp == 1) tc::tmem_alloc(tc::smem_u32(&tmem_base_s), kNB * kN);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base_s;
  const uint32_t idesc = es == 4 ? tc::idesc_tf32(kM, kN) : tc::idesc_bf16(kM, kN);
  volatile int* abort_v = &abort_s;
  const long long lim = P.wait_limit;
  auto give_up = [&]() {
    if (atomicExch(&abort_s, 1) == 0) atomicExch(P.err, 1);
  };
  const int total = P.work.count();
  auto tile_bytes = [&](int ngr, int t) { return (uint32_t)min(8, ngr - 8 * t) * 8u * kp * es; };
  auto group_ptr = [&](int64_t g) { return rows + g * 8 * kp * es; };

  if (warp == 0) {
    // ---- producer: item descriptions one item ahead, then the item's tiles
    if (lane == 0) {
      auto publish = [&](int i) {
        const int r = i % kRing;
        Item d{};
        d.p = -1;
        bool ok = true;
        if (i >= kRing) ok = tc::bar_wait(dempty(r), ((i / kRing) - 1) & 1, abort_v, lim);
        if (!ok) give_up();
        if (ok && !abort_s) d = describe(P, atomicAdd(P.counter, 1), total);
        ring_s[r] = d;
        tc::bar_arrive(dfull(r));                      // release: the description is visible to the waiters
        if (d.p >= 0)
          for (int j = 0; j < min(S, (d.ng + 7) / 8); ++j) tc::bulk_prefetch_l2(group_ptr(d.g0 + 8 * j), tile_bytes(d.ng, j));
        return d;
      };
      uint32_t T = 0;
      Item cur = publish(0);
      for (int i = 0; cur.p >= 0; ++i) {
        const Item nxt = publish(i + 1);
        const int nt = (cur.ng + 7) / 8;
        bool stop = false;
        for (int j = 0; j < nt; ++j, ++T) {
          const uint32_t s = T % S, ph = (T / S) & 1;
          if (j + S < nt) tc::bulk_prefetch_l2(group_ptr(cur.g0 + 8 * (j + S)), tile_bytes(cur.ng, j + S));
          if (!tc::bar_wait(empty(s), ph ^ 1, abort_v, lim)) {
            give_up();
            stop = true;
            break;
          }
          const uint32_t bytes = tile_bytes(cur.ng, j);
          tc::bar_arrive_expect_tx(full(s), bytes);
          tc::bulk_copy_g2s(tc::smem_u32(sB) + s * b_bytes, group_ptr(cur.g0 + 8 * j), bytes, full(s));
          issued_s = (int)(T + 1);
        }
        if (stop) break;
        cur = nxt;
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: never touches an mbarrier (an mbarrier access right
    // after tcgen05.mma stalls the thread until the MMAs drain); the gate
    // hands each tile over through named barrier 2, which also carries stop
    uint32_t T = 0;
    for (;;) {
      if (tc::named_bar_or(2, 64, false)) break;
      const uint32_t s = T % S, b = T % kNB;
      if (lane == 0) {
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(sA) + abuf_s[T & 1] * a_bytes, b0 = tc::smem_u32(sB) + s * b_bytes;
        const int steps = (int)(kp * es / 32);       // one MMA per 32 bytes of K (2 core matrices)
        for (int j = 0; j < steps; ++j) {
          const uint64_t ad = tc::smem_desc(a0 + j * 256, 128, sbo), bd = tc::smem_desc(b0 + j * 256, 128, sbo);
          if constexpr (es == 4) {
            tc::mma_tf32(tmem + b * kN, ad, bd, idesc, j > 0);
          } else {
            tc::mma_bf16(tmem + b * kN, ad, bd, idesc, j > 0);
            tc::mma_bf16(tmem + b * kN, tc::smem_desc(a0 + a_part + j * 256, 128, sbo), bd, idesc, 1);
          }
        }
        tc::mma_commit(empty(s));                      // the stage is free once these MMAs completed
        tc::mma_commit(tfull(b));
      }
      __syncwarp();
      ++T;
      if (lane == 0) committed_s = (int)T;
    }
  } else if (warp == 2) {
    // ---- gate: per item its description and its A buffer, per tile the
    // stage and the accumulator; then it releases the MMA issuer
    uint32_t T = 0;
    bool stopped = false;
    for (int i = 0; !stopped; ++i) {
      int ok = 1, nt = -1;
      if (lane == 0) {
        const int r = i % kRing;
        ok = tc::bar_wait(dfull(r), (i / kRing) & 1, abort_v, lim);
        if (ok) {
          const Item d = ring_s[r];
          nt = d.p < 0 ? -1 : (d.ng + 7) / 8;
        }
        if (ok && nt >= 0) {
          ok = tc::bar_wait(aready(i & 1), (i >> 1) & 1, abort_v, lim);
          if (ok) tc::bar_arrive(agone(i & 1));
        }
        if (!ok) give_up();
      }
      ok = __shfl_sync(kFull, ok, 0);
      nt = __shfl_sync(kFull, nt, 0);
      if (!ok || nt < 0) {
        tc::named_bar_or(2, 64, true);                 // stop the MMA issuer
        break;
      }
      for (int j = 0; j < nt; ++j, ++T) {
        const uint32_t s = T % S, ph = (T / S) & 1, b = T % kNB, tph = (T / kNB) & 1;
        int ok2 = 1;
        if (lane == 0) {
          ok2 = tc::bar_wait(full(s), ph, abort_v, lim) && tc::bar_wait(tempty(b), tph ^ 1, abort_v, lim);
          if (!ok2) give_up();
          else consumed_s = (int)(T + 1);
          abuf_s[T & 1] = (uint32_t)(i & 1);
          tc::fence_before_sync();
        }
        ok2 = __shfl_sync(kFull, ok2, 0);
        if (tc::named_bar_or(2, 64, !ok2)) {
          stopped = true;
          break;
        }
      }
      if (!stopped && lane == 0) tc::bar_arrive(dempty(i % kRing));
    }
  } else {
    // ---- epilogue
    const int m = 32 * (warp & 3) + lane;             // query slot = TMEM lane
    const int jq = 4 * lane + (warp & 3);             // the item's query in that slot
    const int chunks = (int)(kp * es / 16);
    const int64_t qrow = (int64_t)kp * (es == 4 ? 1 : 2);   // elements per query row of Qa
    // stage query qi (or zeros for an idle slot) into row m of A buffer ab
    auto stage_row = [&](int ab, bool use, int64_t qi) {
      unsigned char* arow = sA + ab * a_bytes + (m >> 3) * (kp * 8 * es) + (m & 7) * 16;
      if (use) {
        const ET* q = static_cast<const ET*>(P.Qa) + qi * qrow;
        for (int c = 0; c < chunks; ++c) tc::cp_async16(tc::smem_u32(arow + c * 128), q + (16 / es) * c);
        if constexpr (es == 2)
          for (int c = 0; c < chunks; ++c) tc::cp_async16(tc::smem_u32(arow + a_part + c * 128), q + kp + 8 * c);
      } else {
        for (int c = 0; c < chunks; ++c) {
          *reinterpret_cast<uint4*>(arow + c * 128) = make_uint4(0u, 0u, 0u, 0u);
          if (es == 2) *reinterpret_cast<uint4*>(arow + a_part + c * 128) = make_uint4(0u, 0u, 0u, 0u);
        }
      }
    };
    auto release_a = [&](int ab) {
      tc::cp_async_wait_all();
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) tc::bar_arrive(aready(ab));
    };
    float4* park = park_s + m;                        // [16][kM] the tile's scores by group
    float* cub = list_s + m;                          // [kCap][kM] screened scores
    int32_t* cpos = reinterpret_cast<int32_t*>(list_s + kCap * kM) + m;   // [kCap][kM] padded rows
    // item 0
    Item cur{};
    cur.p = -1;
    int64_t qid_c = 0;
    unsigned gb_c = 0u;
    float qn_c = 0.f, pmax_c = 0.f;
    if (tc::bar_wait(dfull(0), 0, abort_v, lim)) {
      cur = ring_s[0];
      if (cur.p >= 0) {
        const bool use = jq < cur.nqi;
        if (use) {
          qid_c = P.work.query(cur.e0 + jq);
          qn_c = P.qnorm[qid_c];
          gb_c = __ldcg(P.gbound + qid_c);
        }
        pmax_c = P.pmax[cur.p];
        stage_row(0, use, qid_c);
        release_a(0);
      }
    } else {
      give_up();
    }
    uint32_t T = 0;
    for (int i = 0; cur.p >= 0 && !abort_s; ++i) {
      // the next item: its description and its queries' ids now; after this
      // item's first tile (item i - 1's MMAs, the last readers of the other
      // A buffer, have then completed) its queries' norms and bounds, and
      // their rows copied into that buffer, released to the MMA issuer a few
      // tiles later
      Item nxt{};
      nxt.p = -1;
      if (tc::bar_wait(dfull((i + 1) % kRing), ((i + 1) / kRing) & 1, abort_v, lim)) nxt = ring_s[(i + 1) % kRing];
      else give_up();
      const bool has_next = nxt.p >= 0;
      const bool use_n = has_next && jq < nxt.nqi;
      int32_t pv_n = 0;
      float pmax_n = 0.f;
      if (use_n) pv_n = __ldg(P.work.pair_vals + nxt.e0 + jq);
      if (has_next) pmax_n = __ldg(P.pmax + nxt.p);
      int64_t qid_n = 0;
      unsigned gb_n = 0u;
      float qn_n = 0.f;
      bool staged = false, released = false;
      auto stage_next = [&]() {
        if (staged) return;
        staged = true;
        if (!has_next) return;
        if (use_n) {
          qid_n = pv_n / P.work.tmax;
          qn_n = P.qnorm[qid_n];
          gb_n = __ldcg(P.gbound + qid_n);
        }
        stage_row((i + 1) & 1, use_n, qid_n);
      };
      auto release_next = [&]() {
        if (released || !has_next) return;
        released = true;
        // buffer (i + 1) & 1 last held item i - 1: the gate must have seen it
        if (i >= 1 && !tc::bar_wait(agone((i + 1) & 1), ((i - 1) >> 1) & 1, abort_v, lim)) give_up();
        release_a((i + 1) & 1);
      };

      // ---- the current item
      const bool active = jq < cur.nqi;
      const float dlt = P.dscale * qn_c * pmax_c;     // |s~ - exact| < dlt / 2 for every row of p
      float gq = active ? unordered_key(gb_c) - dlt : -INFINITY;
      float gt[kGK];                                  // the 16 largest group maxima, descending
#pragma unroll
      for (int j = 0; j < kGK; ++j) gt[j] = -INFINITY;
      float ak = -INFINITY, cut = gq;
      int cnt = 0, wg = 0;                            // candidates in shared memory / in the pair's global list
      bool ovf = false;
      Cand* out = P.cand + (cur.e0 + (active ? jq : 0)) * (int64_t)kGmList;
      // at the end of the item the shared-memory candidates at or above c_cut
      // move to the pair's global list as (upper bound of the exact score,
      // row); only a full global list overflows (the partition is then
      // rescanned exactly)
      auto flush = [&](float c_cut) {
        for (int j2 = 0; j2 < cnt; ++j2) {
          const float sv = cub[j2 * kM];
          if (sv >= c_cut) {
            if (wg < kGmList) out[wg++] = Cand{sv + dlt, cpos[j2 * kM]};
            else ovf = true;
          }
        }
        cnt = 0;
      };
      const int nt = (cur.ng + 7) / 8;
      for (int j = 0; j < nt; ++j, ++T) {
        const uint32_t b = T % kNB, tph = (T / kNB) & 1;
        const bool ok = tc::bar_wait(tfull(b), tph, abort_v, lim);
        if (!ok) give_up();
        tc::fence_after_sync();
        uint32_t ra[32], rb[32];
        float g[16], gu[16];                          // the tile's group maxima (groups of four or eight rows)
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + b * kN;
        const int nvalid = min(kN, cur.nrows - kN * j);
        // After an item's first two tiles the bound has mostly converged: a
        // full tile then takes eight groups of eight rows, half the sorting
        // and merging (groups of different sizes are still disjoint sets of
        // distinct rows, so the bound stays valid).
        const bool wide = j >= 2 && nvalid == kN;
        if (ok) {
          if (wide) {
#pragma unroll
            for (int q8 = 0; q8 < 8; ++q8) {
              uint32_t* r = q8 < 4 ? ra : rb;
              tc::tmem_ld8_max(taddr + 8 * q8, r + ((8 * q8) & 31), g[q8]);
            }
          } else {
#pragma unroll
            for (int q4 = 0; q4 < 16; ++q4) {
              uint32_t* r = q4 < 8 ? ra : rb;
              tc::tmem_ld4_max(taddr + 4 * q4, r + ((4 * q4) & 31), g[q4]);
            }
          }
          tc::tmem_ld_wait();
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::bar_arrive(tempty(b));
        if (!ok) break;
        if (j == 0) stage_next();
        if (j == kStageAt) release_next();
        // every fourth tile refresh G_q; the load is issued here and used
        // after the tile's screening, so its latency overlaps that work
        const bool refresh = active && (j & 3) == 3;
        const unsigned gload = refresh ? __ldcg(P.gbound + qid_c) : 0u;
        const int32_t pr0 = (int32_t)(cur.row0 + (int64_t)kN * j);   // row-major position of the tile's first row
        if (wide) {
          float gw[8];
#pragma unroll
          for (int q8 = 0; q8 < 8; ++q8) gw[q8] = g[q8];
          // bitonic sort of the eight group maxima, descending
#pragma unroll
          for (int size = 2; size <= 8; size <<= 1)
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1)
#pragma unroll
              for (int i2 = 0; i2 < 8; ++i2) {
                const int j2 = i2 ^ stride;
                if (j2 > i2) {
                  const bool desc = (i2 & size) == 0;
                  const float x = gw[i2], y = gw[j2];
                  gw[i2] = desc ? fmaxf(x, y) : fminf(x, y);
                  gw[j2] = desc ? fminf(x, y) : fmaxf(x, y);
                }
              }
          // the list's last eight against the reversed eight, then half-cleaners
#pragma unroll
          for (int i2 = 8; i2 < 16; ++i2) gt[i2] = fmaxf(gt[i2], gw[15 - i2]);
#pragma unroll
          for (int stride = 8; stride > 0; stride >>= 1)
#pragma unroll
            for (int i2 = 0; i2 < 16; ++i2)
              if ((i2 & stride) == 0) {
                const float x = gt[i2], y = gt[i2 + stride];
                gt[i2] = fmaxf(x, y);
                gt[i2 + stride] = fminf(x, y);
              }
          if constexpr (KX > 0) {
            ak = gt[KX - 1];
          } else {
            ak = INFINITY;
#pragma unroll
            for (int j2 = 0; j2 < kGK; ++j2)
              if (j2 < k) ak = fminf(ak, gt[j2]);
          }
          cut = fmaxf(ak - 2.f * dlt, gq);
          const float cut0 = active ? cut : INFINITY;
          uint32_t gm = 0u;                           // eight-row groups holding a row at or above the cut
#pragma unroll
          for (int q8 = 0; q8 < 8; ++q8) gm |= (g[q8] >= cut0 ? 1u : 0u) << q8;
          if (__any_sync(kFull, gm != 0u)) {
#pragma unroll
            for (int q4 = 0; q4 < 16; ++q4) {         // only the lane's surviving groups are parked
              const uint32_t* r = q4 < 8 ? ra : rb;
              const int o = (4 * q4) & 31;
              if ((gm >> (q4 >> 1)) & 1u)
                park[q4 * kM] = make_float4(__uint_as_float(r[o]), __uint_as_float(r[o + 1]),
                                            __uint_as_float(r[o + 2]), __uint_as_float(r[o + 3]));
            }
            while (gm) {
              const int q8 = __ffs(gm) - 1;
              gm &= gm - 1u;
              const float4 v0 = park[(2 * q8) * kM], v1 = park[(2 * q8 + 1) * kM];
              const int c0 = 8 * q8;
              const float vv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const bool take = vv[u] >= cut0;
                const bool to_s = take && cnt < kCap;
                const bool to_g = take && !to_s && wg < kGmList;
                if (to_s) {
                  cub[cnt * kM] = vv[u];
                  cpos[cnt * kM] = pr0 + c0 + u;
                }
                if (to_g) out[wg] = Cand{vv[u] + dlt, pr0 + c0 + u};
                ovf = ovf || (take && !to_s && !to_g);
                cnt += to_s ? 1 : 0;
                wg += to_g ? 1 : 0;
              }
            }
          }
        } else {
          if (nvalid < kN) {                            // a short last tile: the missing rows count as -inf
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              if (c >= nvalid) ra[c] = 0xff800000u;
              if (c + 32 >= nvalid) rb[c] = 0xff800000u;
            }
#pragma unroll
            for (int q4 = 0; q4 < 16; ++q4) {
              const uint32_t* r = q4 < 8 ? ra : rb;
              const int o = (4 * q4) & 31;
              g[q4] = fmaxf(fmaxf(__uint_as_float(r[o]), __uint_as_float(r[o + 1])),
                            fmaxf(__uint_as_float(r[o + 2]), __uint_as_float(r[o + 3])));
            }
          }
#pragma unroll
          for (int q4 = 0; q4 < 16; ++q4) gu[q4] = g[q4];
          // bitonic sort of the group maxima, descending
#pragma unroll
          for (int size = 2; size <= 16; size <<= 1)
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1)
#pragma unroll
              for (int i2 = 0; i2 < 16; ++i2) {
                const int j2 = i2 ^ stride;
                if (j2 > i2) {
                  const bool desc = (i2 & size) == 0;
                  const float x = g[i2], y = g[j2];
                  g[i2] = desc ? fmaxf(x, y) : fminf(x, y);
                  g[j2] = desc ? fminf(x, y) : fmaxf(x, y);
                }
              }
          // the 16 largest of two descending lists: the pairwise maxima against
          // the reversed list form a bitonic sequence, which half-cleaners sort
#pragma unroll
          for (int i2 = 0; i2 < 16; ++i2) gt[i2] = fmaxf(gt[i2], g[15 - i2]);
#pragma unroll
          for (int stride = 8; stride > 0; stride >>= 1)
#pragma unroll
            for (int i2 = 0; i2 < 16; ++i2)
              if ((i2 & stride) == 0) {
                const float x = gt[i2], y = gt[i2 + stride];
                gt[i2] = fmaxf(x, y);
                gt[i2 + stride] = fminf(x, y);
              }
          if constexpr (KX > 0) {
            ak = gt[KX - 1];
          } else {                                      // gt[k - 1] as the smallest of the first k: gt stays in registers
            ak = INFINITY;
#pragma unroll
            for (int j2 = 0; j2 < kGK; ++j2)
              if (j2 < k) ak = fminf(ak, gt[j2]);
          }
          cut = fmaxf(ak - 2.f * dlt, gq);              // s~ + dlt < max(L_k, G_q)  <=>  s~ < cut
          const float cut0 = active ? cut : INFINITY;
          uint32_t gm = 0u;                             // groups holding a row at or above the cut
#pragma unroll
          for (int q4 = 0; q4 < 16; ++q4) gm |= (gu[q4] >= cut0 ? 1u : 0u) << q4;
          // past the partition's end nothing is a candidate, not even while the
          // cut is still -inf (the padding rows read as -inf)
          if (nvalid < kN) gm &= (1u << ((nvalid + 3) >> 2)) - 1u;
          if (__any_sync(kFull, gm != 0u)) {
            // park the lane's surviving groups, then one trip per such group:
            // its four scores back from shared memory, the rows at or above
            // the cut appended (predicated, no nested branches)
#pragma unroll
            for (int q4 = 0; q4 < 16; ++q4) {         // only the lane's surviving groups are parked
              const uint32_t* r = q4 < 8 ? ra : rb;
              const int o = (4 * q4) & 31;
              if ((gm >> q4) & 1u)
                park[q4 * kM] = make_float4(__uint_as_float(r[o]), __uint_as_float(r[o + 1]),
                                            __uint_as_float(r[o + 2]), __uint_as_float(r[o + 3]));
            }
            while (gm) {
              const int q4 = __ffs(gm) - 1;
              gm &= gm - 1u;
              const float4 v = park[q4 * kM];
              const int c0 = 4 * q4;
              const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                // to the shared list while it has room, then straight to the
                // pair's global list (stores only, nothing read back)
                const bool take = vv[u] >= cut0 && c0 + u < nvalid;
                const bool to_s = take && cnt < kCap;
                const bool to_g = take && !to_s && wg < kGmList;
                if (to_s) {
                  cub[cnt * kM] = vv[u];
                  cpos[cnt * kM] = pr0 + c0 + u;
                }
                if (to_g) out[wg] = Cand{vv[u] + dlt, pr0 + c0 + u};
                ovf = ovf || (take && !to_s && !to_g);
                cnt += to_s ? 1 : 0;
                wg += to_g ? 1 : 0;
              }
            }
          }
        }
        if (refresh) {
          gq = fmaxf(gq, unordered_key(gload) - dlt);
          cut = fmaxf(cut, gq);
        }
      }
      stage_next();                                   // items with fewer tiles
      release_next();
      if (active && !abort_s) {
        const int64_t e = cur.e0 + jq;
        flush(cut);                                   // the candidates still at or above the final cut
        const float Lk = ak - dlt;                    // -inf while fewer than k groups were seen
        P.hdr[e] = make_int2(__float_as_int(Lk), wg | (ovf ? (int)0x80000000 : 0));
        if (Lk > -INFINITY) atomicMax(P.gbound + qid_c, ordered_key(Lk));
      }
      __syncwarp();
      if (lane == 0) tc::bar_arrive(dempty(i % kRing));
      cur = nxt;
      qid_c = qid_n;
      gb_c = gb_n;
      qn_c = qn_n;
      pmax_c = pmax_n;
    }
    tc::cp_async_wait_all();
  }

  // ---- teardown: after an abort, let copies and MMAs in flight land first
  __syncthreads();
  if (abort_s && threadIdx.x == 0) {
    volatile int never = 0;
    for (int T = consumed_s; T < issued_s; ++T) tc::bar_wait(full(T % S), (T / S) & 1, &never);
  }
  if (abort_s && threadIdx.x == 64 && committed_s > 0) {
    volatile int never = 0;
    const int T = committed_s - 1;
    tc::bar_wait(tfull(T % kNB), (T / kNB) & 1, &never);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, kNB * kN);
}

size_t gm_smem_bytes(int kp, int stages, int es) {
  // each of the two A buffers takes kM * kp * 4 bytes (fp32, or bf16 hi and lo); the
  // parking area kN * kM * 4, the candidate lists 2 * kCap * kM * 4
  return 1024 + (size_t)2 * kM * kp * 4 + (size_t)stages * kN * kp * es + (size_t)kN * kM * 4 +
         (size_t)2 * kCap * kM * 4 + (size_t)(2 * stages + 2 * kNB + 2 * kRing + 4) * 8;
}

int gm_pick_stages(int kp, int es) {
  for (int s = kMaxStages; s >= 2; --s)
    if (gm_smem_bytes(kp, s, es) <= 227 * 1024 - 1024) return s;   // room for the static shared variables
  return 0;
}

// the bf16 query operand: per query its hi row bf16(q) and lo row bf16(q - hi)
__global__ void split_queries_bf16(const float* __restrict__ Qf, int64_t n, int kp, __nv_bfloat16* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * kp) return;
  const int64_t q = i / kp;
  const int c = (int)(i - q * kp);
  const float v = Qf[i];
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  out[q * 2 * kp + c] = hi;
  out[q * 2 * kp + kp + c] = __float2bfloat16_rn(v - __bfloat162float(hi));
}

template <typename ET>
void launch_gm(int k, int grid, size_t smem, cudaStream_t s, const GmParams& prm) {
  auto kern = k == 10 ? scan_gm_kernel<ET, 10> : scan_gm_kernel<ET, 0>;
  SOAR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, kThreads, smem, s>>>(prm);
  SOAR_LAUNCHED();
}

}  // namespace

bool scan_gm_usable(const IndexData& ix, int k) {
  const int es = ix.dtype == SOAR_F32 ? 4 : 2;
  return k >= 1 && k <= kGK && gm_pick_stages(ix.tc_kp, es) >= 2;
}

void scan_gm_launch(const IndexData& ix, const IvfWork& work, int grid, const float* Qf, const float* qnorm,
                    int64_t nq, int k, float dscale, long long wait_limit, int* counter, int* err,
                    unsigned* gbound, Cand* lists, int2* hdr, cudaStream_t s, Scratch& scr) {
  const int es = ix.dtype == SOAR_F32 ? 4 : 2;
  const int stages = gm_pick_stages(ix.tc_kp, es);
  if (k < 1 || k > kGK || stages < 2) fail(SOAR_EUNSUPPORTED, "group-maxima scan: unsupported k or row width");
  const void* Qa = Qf;
  if (es == 2) {
    __nv_bfloat16* qhl = scr.get<__nv_bfloat16>((size_t)nq * 2 * ix.tc_kp);
    const int64_t n = nq * ix.tc_kp;
    split_queries_bf16<<<ceil_div(n, 256), 256, 0, s>>>(Qf, nq, ix.tc_kp, qhl);
    SOAR_LAUNCHED();
    Qa = qhl;
  }
  GmParams prm{work, ix.tc_rows, ix.tc_gstart, ix.tc_pmax, Qa, qnorm, ix.tc_kp, dscale, k, stages, wait_limit,
               counter, err, gbound, lists, hdr};
  const size_t smem = gm_smem_bytes(ix.tc_kp, stages, es);
  if (es == 4) launch_gm<float>(k, grid, smem, s, prm);
  else launch_gm<__nv_bfloat16>(k, grid, smem, s, prm);
}

}  // namespace soar
