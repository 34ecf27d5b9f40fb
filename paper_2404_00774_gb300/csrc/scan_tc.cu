// Batched IVF partition scan on the 5th-generation tensor cores (tcgen05).
//
// One persistent CTA per SM takes work items (partition p, up to 128 of the
// queries that probe p).  The item's queries form the A operand (M = 128
// rows in shared memory, K-major core-matrix layout); the partition's rows
// stream through a 4-stage shared-memory ring as B tiles of 64 rows, copied
// by cp.async.bulk straight from the index, which stores every partition in
// that same layout.  Per tile one thread issues one tcgen05.mma per 32 bytes
// of K (kind::tf32 for an fp32 index, kind::f16 with bf16 operands for a
// bf16 index) into one of four TMEM accumulators (128 lanes x 64 columns,
// so the MMAs run up to three tiles ahead of the epilogue);
// four epilogue warps read the scores back (lane = query).
//
// Screening.  kind::tf32 truncates each fp32 operand to 10 mantissa bits,
// so a screened score s~ lies within 2^-9 ||q|| ||x|| of the fp32 dot
// product (fp32 accumulation error is far below that).  For a bf16 index
// the rows enter exactly and the fp32 query enters as two bf16 terms, q_hi =
// bf16(q) and q_lo = bf16(q - q_hi), in two MMAs into the same accumulator:
// the dropped part is below 2^-18 |q_k| per element, and with the fp32
// accumulation of 2K products and the fp32 rounding of the exact score the
// screened score lies within (2^-18 + 2.5 K 2^-23) ||q|| ||x|| of it, so the
// band delta = max(2^-12, 4 (2^-18 + 2.5 K 2^-23)) ||q|| max_p ||x|| (at
// least a factor 2.9 for K <= 128) is 16 times narrower than the tf32 one;
// on data with tight clusters that keeps the candidate lists short.  Per work item the
// kernel uses one bound delta = 2^-8 ||q|| max_p ||x|| (max over the
// partition's rows: a factor-2 margin).  Per (query, partition) it keeps
//   * the k best screened scores; with a_k the k-th of them,
//     L_k = a_k - delta bounds the partition's k-th best exact score from
//     below, and
//   * the rows with s~ + delta >= L_k (up to kCand, pruned as a_k rises);
//     a row outside that set cannot be in the top k.
// No row is rescored here.  The finishing kernels of finish_tc.cu
// (finish_queries for k <= 32; rescore_wide and the merge for k > 32) later
// take, per query, the largest L_k over its partitions, rescore exactly the
// candidates whose upper bound reaches it and rescan exactly any partition
// whose candidate list overflowed, so the results equal those of an exact
// scan.
//
// Warp roles: 0 = bulk-copy producer (it also claims and resolves the next
// work item ahead and prefetches its first tiles into L2), 1 = TMEM owner and
// MMA issuer, 2 = gate (does the mbarrier waits for the MMA issuer), 3..6 =
// epilogue (query slot = 32 * (warp % 4) + lane, its TMEM lane).  A stage of
// the tile ring is released by the MMA's completion, not by the epilogue.
// Every mbarrier wait is bounded (about a second); on expiry the CTA raises
// *err, stops taking work, waits (bounded) for its copies and MMAs in flight,
// frees its TMEM and returns.
#include "scan_common.cuh"
#include "tc.cuh"

namespace soar {

namespace {

constexpr int kM = 128;        // query slots per item (MMA M)
constexpr int kN = 64;         // rows per tile (MMA N)
constexpr int kThreads = 224;  // producer, MMA issuer, gate, 4 epilogue warps
constexpr int kMaxStages = 4;
constexpr int kNB = 4;         // TMEM accumulator buffers (kN columns each)
constexpr int kCand = 32;      // candidate rows kept per (query, partition), register mode
constexpr int kWideK = kTcWideK;   // largest k of the heap mode
constexpr int kWideList = kTcWideList;   // largest global candidate list of the heap mode

// Candidate-list length per (query, partition) slot: kGmList for k <= 16
// (the group-maxima scan of scan_gm.cu appends without a final filter),
// kCand for k <= 32, else 2k rounded up to a warp multiple (room to append
// between compactions).
__host__ __device__ constexpr int list_len_for(int k) {
  return k <= 16 ? kGmList
                 : k <= kCand ? kCand
                              : ((2 * k + 31) / 32 * 32 > kWideList ? kWideList : (2 * k + 31) / 32 * 32);
}

// Shared memory behind the tile scores: register mode keeps kCand candidates
// (score, padded row) per query slot, heap mode a min-heap of k scores.
__host__ __device__ constexpr size_t ext_bytes(int k) {
  return k <= kCand ? (size_t)kM * kCand * 8 : (size_t)kM * k * 4;
}

struct TcParams {
  IvfWork work;
  const void* rows;        // index rows (fp32 or bf16), core-matrix layout, 8-row groups
  const int64_t* gstart;   // [c + 1] first 8-row group of each partition
  const float* pmax;       // [c] largest ||x|| of each partition
  const float* Qf;         // [nq][kp] fp32 query rows
  const float* qnorm;      // [nq]
  int kp;                  // K, a multiple of 8
  float dscale;            // delta / (||q|| max_p ||x||)
  int k;                   // top-k length
  int kc;                  // candidate-list capacity per pair slot
  int stages;
  long long wait_limit;    // SM cycles a pipeline wait may take before the CTA gives up
  int* counter;            // work-item counter
  int* err;                // set to 1 when a wait expired
  unsigned* gbound;        // [nq] per-query lower bound of the final k-th best exact score (ordered key)
  Cand* cand;              // [pairs][kc] (ub, row-major row position) candidates
  int2* hdr;               // [pairs] (L_k as float bits, count | overflow << 31)
};

__device__ __forceinline__ unsigned ordered(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unordered(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// A work item resolved: partition p (-1: no more items), its first pair slot
// and query count, its row count, first 8-row group and group count.
struct ItemDesc {
  int p, nqi, nrows, ng;
  int64_t e0, g0, row0;
};

__device__ ItemDesc describe_item(const TcParams& P, int item, int total) {
  ItemDesc d{};
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

// KMAX > 0: register top-k of up to KMAX entries (EXACT: k == KMAX known at
// compile time, which makes every top-k insertion a fixed compare-exchange
// chain); KMAX == 0: heap mode.
template <typename ET, int KMAX, bool EXACT>
__global__ void __launch_bounds__(kThreads, 1) scan_tc_kernel(TcParams P) {
  constexpr uint32_t es = sizeof(ET);            // bytes per operand element
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned carve-up of the dynamic shared memory
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int kp = P.kp, k = EXACT ? KMAX : P.k, S = P.stages;
  const uint32_t sbo = (uint32_t)kp * 8u * es;        // bytes between 8-row groups
  const uint32_t a_bytes = (uint32_t)kM * kp * es;     // one part (bf16: hi, then lo)
  const uint32_t b_bytes = (uint32_t)kN * kp * es;
  const char* rows = static_cast<const char*>(P.rows);
  unsigned char* sA = base;
  unsigned char* sB = base + (es == 4 ? 1 : 2) * a_bytes;
  float* av_s = reinterpret_cast<float*>(sB + (size_t)S * b_bytes);  // [kN][kM] parked scores
  // per-slot arrays are interleaved slot-fastest ([entry][kM]) so that the 32
  // lanes of a warp always touch 32 distinct banks
  float* ext_s = av_s + kN * kM;   // candidates [kCand][kM] (+ rows) or the heap [k][kM]
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(ext_s) + ext_bytes(k));
  // bars: full[S], empty[S], tfull[kNB], tempty[kNB]
  __shared__ uint32_t tmem_base_s;
  __shared__ ItemDesc item_s;
  __shared__ int abort_s;
  __shared__ int issued_s, consumed_s, committed_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int s) { return tc::smem_u32(&bars[s]); };
  auto empty = [&](int s) { return tc::smem_u32(&bars[S + s]); };
  auto tfull = [&](int b) { return tc::smem_u32(&bars[2 * S + b]); };
  auto tempty = [&](int b) { return tc::smem_u32(&bars[2 * S + kNB + b]); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::bar_init(full(s), 1);
      tc::bar_init(empty(s), 1);
    }
    for (int b = 0; b < kNB; ++b) {
      tc::bar_init(tfull(b), 1);
      tc::bar_init(tempty(b), 4);
    }
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
  auto give_up = [&]() {
    if (atomicExch(&abort_s, 1) == 0) atomicExch(P.err, 1);
  };
  // epilogue thread: the TMEM lane quarter of warp % 4 holds query slot m;
  // it takes the item's query j = 4 * lane + warp % 4, so that the active
  // queries spread evenly over the four epilogue warps
  const int m = 32 * (warp & 3) + lane;
  const int jq = 4 * lane + (warp & 3);

  uint32_t tile_ctr = 0, committed = 0;
  const int total = P.work.count();
  // The producer thread claims items one ahead and resolves the next item's
  // description (a chain of dependent global loads: a binary search over the
  // item table, then the partition's offsets) while the current item runs;
  // the other threads read it from shared memory at the item boundary.
  ItemDesc next{};
  if (threadIdx.x == 0) next = describe_item(P, atomicAdd(P.counter, 1), total);
  for (;;) {
    if (threadIdx.x == 0) {
      item_s = next;
      if (abort_s) item_s.p = -1;
    }
    __syncthreads();
    const ItemDesc D = item_s;
    if (D.p < 0) break;
    const int p = D.p;
    const int64_t e0 = D.e0;
    const int nqi = D.nqi;
    const int nrows = D.nrows;
    const int64_t g0 = D.g0;
    const int ng = D.ng;
    const int ntiles = (ng + 7) / 8;

    // ---- queries of the item -> A operand (row m of the epilogue threads),
    // staged by 16-byte cp.async so that the row's loads are all in flight
    // at once; the producer warp is not held by this barrier and already
    // streams the item's tiles.  The epilogue's per-slot inputs (query id,
    // its published bound, its norm, the partition's largest row norm) are
    // loaded meanwhile, off the first tile's critical path.
    int64_t qid_pre = 0;
    unsigned gb_pre = 0u;
    float qn_pre = 0.f, pmax_pre = 0.f;
    if (warp >= 3) {
      // row m's 16-byte chunk c sits at (m / 8) * 8 K es + c * 128 + (m % 8) * 16
      unsigned char* arow = sA + (m >> 3) * (kp * 8 * es) + (m & 7) * 16;
      const int chunks = (int)(kp * es / 16);
      pmax_pre = P.pmax[p];
      if (jq < nqi) {
        const int64_t qi = P.work.query(e0 + jq);
        const float* q = P.Qf + qi * (int64_t)kp;
        if constexpr (es == 4) {
          for (int c = 0; c < chunks; ++c) tc::cp_async16(tc::smem_u32(arow + c * 128), q + 4 * c);
        } else {
          // bf16 operands: the fp32 query as hi = bf16(q) (first A part) and
          // lo = bf16(q - hi) (second A part), 8 elements per chunk
          for (int c = 0; c < chunks; ++c) {
            const float4 a0 = __ldg(reinterpret_cast<const float4*>(q + 8 * c));
            const float4 a1 = __ldg(reinterpret_cast<const float4*>(q + 8 * c + 4));
            const float v[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const __nv_bfloat162 bh = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);
              const float2 fh = __bfloat1622float2(bh);
              const __nv_bfloat162 bl = __floats2bfloat162_rn(v[2 * h] - fh.x, v[2 * h + 1] - fh.y);
              hi[h] = *reinterpret_cast<const uint32_t*>(&bh);
              lo[h] = *reinterpret_cast<const uint32_t*>(&bl);
            }
            *reinterpret_cast<uint4*>(arow + c * 128) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(arow + a_bytes + c * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
        qid_pre = qi;
        qn_pre = P.qnorm[qi];
        gb_pre = __ldcg(P.gbound + qi);
      } else {
        for (int c = 0; c < chunks; ++c) {
          *reinterpret_cast<uint4*>(arow + c * 128) = make_uint4(0u, 0u, 0u, 0u);
          if (es == 2) *reinterpret_cast<uint4*>(arow + a_bytes + c * 128) = make_uint4(0u, 0u, 0u, 0u);
        }
      }
      tc::cp_async_wait_all();
      tc::fence_async_smem();
    }
    if (warp > 0) asm volatile("bar.sync 3, %0;" ::"n"(kThreads - 32) : "memory");

    if (warp == 0) {
      // ---- producer: one thread streams the partition's tiles, keeping the
      // tiles S ahead of the copies in flight prefetched into L2
      if (lane == 0) {
        auto tile_bytes = [&](int ngr, int t) { return (uint32_t)min(8, ngr - 8 * t) * 8u * kp * es; };
        auto group_ptr = [&](int64_t g) { return rows + g * 8 * kp * es; };
        for (int i = 0; i < min(S, ntiles); ++i) tc::bulk_prefetch_l2(group_ptr(g0 + 8 * i), tile_bytes(ng, i));
        for (int i = 0; i < ntiles; ++i) {
          const uint32_t T = tile_ctr + i, s = T % S, ph = (T / S) & 1;
          if (i + S < ntiles) tc::bulk_prefetch_l2(group_ptr(g0 + 8 * (i + S)), tile_bytes(ng, i + S));
          if (!tc::bar_wait(empty(s), ph ^ 1, abort_v, P.wait_limit)) { give_up(); break; }
          const uint32_t bytes = tile_bytes(ng, i);
          tc::bar_arrive_expect_tx(full(s), bytes);
          tc::bulk_copy_g2s(tc::smem_u32(sB) + s * b_bytes, group_ptr(g0 + 8 * i), bytes, full(s));
          issued_s = (int)(T + 1);
        }
        // claim the next item, resolve it and warm L2 with its first tiles
        next = describe_item(P, atomicAdd(P.counter, 1), total);
        if (next.p >= 0)
          for (int i = 0; i < min(S, (next.ng + 7) / 8); ++i)
            tc::bulk_prefetch_l2(group_ptr(next.g0 + 8 * i), tile_bytes(next.ng, i));
      }
    } else if (warp == 1) {
      // ---- MMA issuer.  It never touches an mbarrier (an mbarrier access
      // right after tcgen05.mma stalls the thread until the MMAs drain): the
      // gate warp waits for it and hands each tile over through a named
      // barrier that also carries the stop flag.
      for (int i = 0; i < ntiles; ++i) {
        if (tc::named_bar_or(2, 64, false)) break;
        const uint32_t T = tile_ctr + i, s = T % S, b = T % kNB;
        if (lane == 0) {
          tc::fence_after_sync();
          const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB) + s * b_bytes;
          const int steps = (int)(kp * es / 32);   // one MMA per 32 bytes of K (2 core matrices)
          for (int j = 0; j < steps; ++j) {
            const uint64_t ad = tc::smem_desc(a0 + j * 256, 128, sbo), bd = tc::smem_desc(b0 + j * 256, 128, sbo);
            if constexpr (es == 4) {
              tc::mma_tf32(tmem + b * kN, ad, bd, idesc, j > 0);
            } else {
              tc::mma_bf16(tmem + b * kN, ad, bd, idesc, j > 0);
              tc::mma_bf16(tmem + b * kN, tc::smem_desc(a0 + a_bytes + j * 256, 128, sbo), bd, idesc, 1);
            }
          }
          tc::mma_commit(empty(s));                  // the stage is free once these MMAs completed
          tc::mma_commit(tfull(b));
        }
        __syncwarp();
        committed = T + 1;
      }
      if (lane == 0) committed_s = (int)committed;
    } else if (warp == 2) {
      // ---- gate: waits for each tile's stage and TMEM buffer, then releases
      // the MMA issuer
      for (int i = 0; i < ntiles; ++i) {
        const uint32_t T = tile_ctr + i, s = T % S, ph = (T / S) & 1, b = T % kNB, tph = (T / kNB) & 1;
        int ok = 1;
        if (lane == 0) {
          ok = tc::bar_wait(full(s), ph, abort_v, P.wait_limit) &&
               tc::bar_wait(tempty(b), tph ^ 1, abort_v, P.wait_limit);
          if (!ok) give_up();
          else consumed_s = (int)(T + 1);
          tc::fence_before_sync();
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (tc::named_bar_or(2, 64, !ok)) break;
      }
    } else {
      // ---- epilogue: screening bounds and candidate rows per query
      const bool active = jq < nqi;
      const float dlt = P.dscale * qn_pre * pmax_pre;   // |s~ - exact| < dlt / 2 for every row of p
      // G_q, published by this query's finished partitions, bounds its final
      // k-th best exact score from below: rows with s~ + dlt < G_q cannot count
      const int64_t qid = qid_pre;
      float gq = active ? unordered(gb_pre) - dlt : -INFINITY;
      float ak = -INFINITY;                            // k-th best screened score (-inf until k seen)
      float floor_ = -INFINITY;                        // a lower bound of the k-th best screened score
      float cut = gq;                                  // rows below cut cannot reach the top k
      int cnt = 0;
      bool ovf = false;
      // register mode (KMAX > 0): the k best screened scores in the last k
      // of KMAX registers (the first KMAX - k hold +inf, which no insertion
      // passes, so the k-th best is always the last register) and up to
      // kCand candidates in shared memory.  Heap mode (KMAX == 0): the k best
      // screened scores in a shared-memory min-heap and up to kc candidates
      // in the slot's global list.
      float ta[KMAX > 0 ? KMAX : 1];
#pragma unroll
      for (int j = 0; j < (KMAX > 0 ? KMAX : 1); ++j) ta[j] = j < KMAX - k ? INFINITY : -INFINITY;
      float* cub = ext_s + m;                                              // [kCand][kM] scores
      int32_t* cpos = reinterpret_cast<int32_t*>(ext_s + kM * kCand) + m;   // [kCand][kM] padded rows
      float* heap = ext_s + m;                                             // heap mode: [k][kM]
      int hn = 0;
      Cand* glist = P.cand + (e0 + (active ? jq : 0)) * (int64_t)P.kc;     // heap mode candidates
      for (int i = 0; i < ntiles; ++i) {
        const uint32_t T = tile_ctr + i, b = T % kNB, tph = (T / kNB) & 1;
        const bool ok = tc::bar_wait(tfull(b), tph, abort_v, P.wait_limit);
        if (!ok) give_up();
        tc::fence_after_sync();
        uint32_t r0[32], r1[32];
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + b * kN;
        if (ok) {
          tc::tmem_ld32(taddr, r0);
          tc::tmem_ld32(taddr + 32, r1);
          tc::tmem_ld_wait();
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::bar_arrive(tempty(b));
        if (!ok) break;
        // every fourth tile refresh G_q; the load is issued here and used
        // after the tile's screening, so its latency overlaps that work
        const bool refresh = active && (i & 3) == 3;
        const unsigned gload = refresh ? __ldcg(P.gbound + qid) : 0u;
        const int nvalid = min(kN, nrows - kN * i);
        const int32_t pr0 = (int32_t)(D.row0 + (int64_t)kN * i);   // row-major position of the tile's first row
        if (KMAX > 0 && ak == -INFINITY && floor_ == -INFINITY && k <= 16 && nvalid == kN) {
          // the k-th largest of 16 group maxima (groups of 4 rows) is a lower
          // bound of the tile's k-th best screened score: seed the cut with it
          float g[16];
#pragma unroll
          for (int q4 = 0; q4 < 16; ++q4) {
            const int c = 4 * q4;
            const float a0 = __uint_as_float(c < 32 ? r0[c & 31] : r1[c & 31]);
            const float a1 = __uint_as_float(c + 1 < 32 ? r0[(c + 1) & 31] : r1[(c + 1) & 31]);
            const float a2 = __uint_as_float(c + 2 < 32 ? r0[(c + 2) & 31] : r1[(c + 2) & 31]);
            const float a3 = __uint_as_float(c + 3 < 32 ? r0[(c + 3) & 31] : r1[(c + 3) & 31]);
            g[q4] = fmaxf(fmaxf(a0, a1), fmaxf(a2, a3));
          }
          // bitonic sort of the 16 maxima, descending
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
          // the k-th largest = the smallest of the first k (g is sorted)
          float seed = INFINITY;
#pragma unroll
          for (int j2 = 0; j2 < 16; ++j2)
            if (j2 < k) seed = fminf(seed, g[j2]);
          floor_ = seed;
          cut = fmaxf(seed - 2.f * dlt, gq);
        }
        // register-only screen against the cut at the tile's start (the cut
        // only rises, so this keeps a superset); survivors parked in smem.
        // An idle slot screens against +inf; the bits of a short last tile's
        // missing rows are cleared afterwards.  Four independent 16-column
        // masks keep the OR chains short.
        const float cut0 = active ? cut : INFINITY;
        uint32_t mq[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int c = 0; c < kN; ++c) {
          const float a = __uint_as_float(c < 32 ? r0[c & 31] : r1[c & 31]);
          if (a >= cut0) {
            mq[c >> 4] |= 1u << (c & 31);
            av_s[c * kM + m] = a;
          }
        }
        uint64_t mask = (uint64_t)(mq[0] | mq[1]) | ((uint64_t)(mq[2] | mq[3]) << 32);
        if (nvalid < kN) mask &= ((uint64_t)1 << nvalid) - 1;
        // one pass over the survivors in row order: each raises the k best
        // screened scores, then joins the candidates if it still reaches the
        // (risen) cut; the item's final cut filters the list at the end
        auto survivor = [&](const int c, const float a) {
          if (a < cut) return;
          if constexpr (KMAX > 0) {
            if (a > ak) {
              float v = a;
#pragma unroll
              for (int j = 0; j < KMAX; ++j) {
                const float hi = fmaxf(ta[j], v);
                v = fminf(ta[j], v);
                ta[j] = hi;
              }
              ak = ta[KMAX > 0 ? KMAX - 1 : 0];
            }
          } else {
            if (hn < k) {                            // heap not full: sift the new score up
              int j = hn++;
              while (j > 0) {
                const int par = (j - 1) >> 1;
                const float pv = heap[par * kM];
                if (pv <= a) break;
                heap[j * kM] = pv;
                j = par;
              }
              heap[j * kM] = a;
              if (hn == k) ak = heap[0];
            } else if (a > ak) {                     // replace the minimum, sift down
              int j = 0;
              for (;;) {
                int ch = 2 * j + 1;
                if (ch >= k) break;
                float cv = heap[ch * kM];
                if (ch + 1 < k) {
                  const float c2 = heap[(ch + 1) * kM];
                  if (c2 < cv) { cv = c2; ++ch; }
                }
                if (cv >= a) break;
                heap[j * kM] = cv;
                j = ch;
              }
              heap[j * kM] = a;
              ak = heap[0];
            }
          }
          cut = fmaxf(fmaxf(ak, floor_) - 2.f * dlt, gq);   // s~ + dlt < max(L_k, G_q)  <=>  s~ < cut
          if (a < cut) return;
          if constexpr (KMAX > 0) {
            if (cnt == kCand) {                      // drop candidates that fell below the cut
              int w = 0;
              for (int j = 0; j < kCand; ++j)
                if (cub[j * kM] >= cut) { cub[w * kM] = cub[j * kM]; cpos[w * kM] = cpos[j * kM]; ++w; }
              cnt = w;
            }
            if (cnt < kCand) {
              cub[cnt * kM] = a;
              cpos[cnt * kM] = pr0 + c;
              ++cnt;
            } else {
              ovf = true;
            }
          } else {
            if (cnt == P.kc) {                       // drop candidates that fell below the cut
              int w = 0;
              for (int j = 0; j < P.kc; ++j) {
                const Cand v = glist[j];
                if (v.s >= cut) glist[w++] = v;
              }
              cnt = w;
            }
            if (cnt < P.kc) glist[cnt++] = Cand{a, pr0 + c};
            else ovf = true;
          }
        };
        for (; mask; mask &= mask - 1) {
          const int c = __ffsll((long long)mask) - 1;
          survivor(c, av_s[c * kM + m]);
        }
        if (refresh) {
          gq = fmaxf(gq, unordered(gload) - dlt);
          cut = fmaxf(cut, gq);
        }
      }
      if (active && !abort_s) {
        const int64_t e = e0 + jq;
        int w = 0;
        if constexpr (KMAX > 0) {
          Cand* out = P.cand + e * (int64_t)P.kc;
          for (int j = 0; j < cnt; ++j)
            if (cub[j * kM] >= cut) out[w++] = Cand{cub[j * kM] + dlt, cpos[j * kM]};   // upper bound of the exact score
        } else {
          for (int j = 0; j < cnt; ++j) {
            const Cand v = glist[j];
            if (v.s >= cut) glist[w++] = Cand{v.s + dlt, v.id};
          }
        }
        const float Lk = fmaxf(ak, floor_) - dlt;   // -inf while fewer than k rows were seen
        P.hdr[e] = make_int2(__float_as_int(Lk), w | (ovf ? (int)0x80000000 : 0));
        if (Lk > -INFINITY) atomicMax(P.gbound + qid, ordered(Lk));
      }
    }
    tile_ctr += ntiles;
    __syncthreads();
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

size_t smem_bytes(int kp, int k, int stages, int es) {
  // the A operand takes kM * kp * 4 bytes either way (fp32, or bf16 hi and lo)
  return 1024 + (size_t)kM * kp * 4 + (size_t)stages * kN * kp * es + (size_t)kN * kM * 4 + ext_bytes(k) +
         (size_t)(2 * stages + 2 * kNB) * 8;
}

// delta / (||q|| max_p ||x||) of the screen (see the header comment)
float delta_scale(int kp, int es) {
  if (es == 4) return 1.f / 256.f;
  return std::max(1.f / 4096.f, 4.f * (std::ldexp(1.f, -18) + 2.5f * kp * std::ldexp(1.f, -23)));
}

int pick_stages(int kp, int k, int es) {
  for (int s = kMaxStages; s >= 2; --s)
    if (smem_bytes(kp, k, s, es) <= 227 * 1024 - 1024) return s;   // room for the static shared variables
  return 0;
}

template <typename ET>
void launch_scan_tc(int k, int grid, size_t smem, cudaStream_t s, const TcParams& prm) {
  auto kern = k == 10   ? scan_tc_kernel<ET, 10, true>
              : k <= 16 ? scan_tc_kernel<ET, 16, false>
              : k <= kCand ? scan_tc_kernel<ET, 32, false> : scan_tc_kernel<ET, 0, false>;
  SOAR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, kThreads, smem, s>>>(prm);
  SOAR_LAUNCHED();
}


__global__ void fill_u32(unsigned* __restrict__ a, int64_t n, unsigned v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

// Every pair slot's header before the scan: bound -inf, no candidates, so
// that a slot the scan never wrote (a CTA that gave up a wait) is read by the
// finishing kernels as an empty list.
__global__ void clear_headers(int2* __restrict__ hdr, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) hdr[i] = make_int2(__float_as_int(-INFINITY), 0);
}

std::atomic<long long> g_wait_limit{0};

}  // namespace

void set_scan_wait_limit(long long cycles) { g_wait_limit.store(cycles > 0 ? cycles : 0); }

int scan_tc_max_k(const IndexData& ix) {
  const int es = ix.dtype == SOAR_F32 ? 4 : 2;
  int k = 0;
  while (k < kWideK && pick_stages(ix.tc_kp, k + 1, es) >= 2) ++k;
  return k;
}

int scan_tc_list_len(int k) { return list_len_for(k); }

bool scan_tc_search(const IndexData& ix, const IvfWork& work, int max_items, const float* Qf, const float* qnorm,
                    const int32_t* top, const int32_t* inv, const int32_t* tpq, int64_t nq, int t, int k,
                    Cand* lists, int* err, int64_t* ids_out, float* scores_out, cudaStream_t s, Scratch& scr) {
  const int es = ix.dtype == SOAR_F32 ? 4 : 2;
  const int stages = pick_stages(ix.tc_kp, k, es);
  if (stages < 2 || k > kWideK) fail(SOAR_EUNSUPPORTED, "tensor-core scan: k too large");
  const int kc = list_len_for(k);
  const int64_t P = nq * t;
  int2* hdr = scr.get<int2>(P);
  clear_headers<<<ceil_div(P, 256), 256, 0, s>>>(hdr, P);
  SOAR_LAUNCHED();
  const long long lim = g_wait_limit.load();
  TcParams prm{work, ix.tc_rows, ix.tc_gstart, ix.tc_pmax, Qf, qnorm, ix.tc_kp, delta_scale(ix.tc_kp, es), k, kc,
               stages, lim > 0 ? lim : tc::kWaitLimit, nullptr, err, nullptr, lists, hdr};
  prm.gbound = scr.get<unsigned>(nq);
  fill_u32<<<ceil_div(nq, 256), 256, 0, s>>>(prm.gbound, nq, 0x007fffffu);   // ordered key of -inf
  SOAR_LAUNCHED();
  prm.counter = scr.get<int>(1);
  SOAR_CUDA(cudaMemsetAsync(prm.counter, 0, sizeof(int), s));
  const size_t smem = smem_bytes(ix.tc_kp, k, stages, es);
  const int grid = std::max(1, std::min(max_items, num_sms()));
  stage_mark(s, "scan", true);
  if (scan_gm_usable(ix, k))
    scan_gm_launch(ix, work, grid, Qf, qnorm, nq, k, prm.dscale, prm.wait_limit, prm.counter, err, prm.gbound,
                   lists, hdr, s, scr);
  else if (es == 4)
    launch_scan_tc<float>(k, grid, smem, s, prm);
  else
    launch_scan_tc<__nv_bfloat16>(k, grid, smem, s, prm);
  stage_mark(s, "scan", false);
  stage_mark(s, "rescore", true);
  if (k <= kCand) {
    finish_tc_queries(ix, lists, hdr, inv, nq, t, tpq, Qf, top, k, kc, ids_out, scores_out, s);
    stage_mark(s, "rescore", false);
    return true;
  }
  rescore_tc_wide(ix, lists, hdr, inv, work.pair_vals, nq, t, tpq, Qf, top, k, kc, s, scr);
  stage_mark(s, "rescore", false);
  return false;
}

}  // namespace soar
