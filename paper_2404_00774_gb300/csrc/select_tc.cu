// Partition selection on the 5th-generation tensor cores (tcgen05): the
// probing step of an IVF search (Section 2.2), in which a query is scored
// against every centroid by inner product and the t best partitions are
// searched.  One kernel computes the scores and keeps each query's t best,
// so the nq x c score matrix never exists.
//
// Precision.  kind::tf32 keeps 10 explicit mantissa bits of each operand, so
// every fp32 value v enters as two tf32 values, hi = v rounded to tf32 and
// lo = (v - hi) rounded to tf32, and the kernel accumulates
//     q.c = q_hi.c_hi + q_hi.c_lo + q_lo.c_hi
// in three MMA passes into one fp32 TMEM accumulator.  Per term the dropped
// parts (q_lo c_lo and the roundings of lo) are below 3 * 2^-22 |q_k c_k|,
// so a score's error stays below 2^-20 sum_k |q_k c_k| plus the fp32
// accumulation: the accuracy of a fp32 dot product (whose worst case over
// K terms is K * 2^-24 sum_k |q_k c_k|).
//
// Layout.  The index keeps the codebook packed for this kernel at build
// time: tiles of 64 centroids (zero rows past c), each tile the hi part then
// the lo part, both in the K-major core-matrix layout of tc.cuh, so one
// contiguous bulk copy moves a tile.  The CTA's 128 queries are split into
// hi / lo in shared memory by the epilogue warps before the first MMA.
//
// Warp roles as in the partition scan: 0 = bulk-copy producer (2-stage ring),
// 1 = TMEM owner and MMA issuer, 2 = gate (does the mbarrier waits for the
// MMA issuer, which would stall on an mbarrier access right after its MMAs),
// 3..6 = epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, one query per
// lane.  Each epilogue thread keeps its query's t best (score, id) in
// registers; a tile's 64 scores are screened 16 at a time against the
// current t-th best, the survivors parked in shared memory and inserted.
// Columns arrive in ascending id order and only a strictly larger score is
// inserted, so equal scores keep the lower centroid id first (the order of
// the other selection kernels: score descending, id ascending).
// Every mbarrier wait is bounded (about a second); on expiry the CTA raises
// *err, stops, waits (bounded) for its copies and MMAs in flight, frees its
// TMEM and returns.
#include "internal.cuh"
#include "tc.cuh"

namespace soar {

namespace {

constexpr int kM = 128;        // queries per CTA (MMA M)
constexpr int kN = 64;         // centroids per tile (MMA N)
constexpr int kThreads = 224;  // producer, MMA issuer, gate, 4 epilogue warps
constexpr int kStages = 2;
constexpr int kChunk = 16;     // columns screened per survivor pass

// v rounded to the nearest value with 10 explicit mantissa bits (ties away
// from zero); infinities and NaNs pass through.
__device__ __forceinline__ float round_tf32(float v) {
  uint32_t u = __float_as_uint(v);
  if ((u & 0x7f800000u) == 0x7f800000u) return v;
  u = (u + 0x1000u) & 0xffffe000u;
  return __uint_as_float(u);
}

// Element (r, k) of a K-major core-matrix operand with kp columns (tc.cuh).
__device__ __forceinline__ int64_t core_offset(int r, int k, int kp) {
  return (int64_t)(r >> 3) * (8 * kp) + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

// Packs C [c][d] into tiles of 64 rows: [tile][hi, lo][64 x kp core layout].
__global__ void pack_codebook_split(const float* __restrict__ C, int c, int d, int kp, int tiles,
                                     float* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)tiles * kN * kp) return;
  const int k = (int)(idx % kp);
  const int64_t r = idx / kp;
  const int tile = (int)(r / kN), rr = (int)(r % kN);
  const float v = (r < c && k < d) ? C[r * d + k] : 0.f;
  const float hi = round_tf32(v);
  const float lo = round_tf32(v - hi);
  float* base = out + (int64_t)tile * 2 * kN * kp;
  const int64_t off = core_offset(rr, k, kp);
  base[off] = hi;
  base[(int64_t)kN * kp + off] = lo;
}

struct SelParams {
  const float* Qf;    // [nq][qstride] fp32 queries, columns >= d ignored
  int64_t nq;
  int qstride, d, kp;
  const float* cb;    // packed codebook
  int c, tiles, t;
  int32_t* top;       // [nq][t]
  float* top_s;       // [nq][t] or null
  int* err;           // set to 1 when a wait expired
};

template <int TMAX>
__global__ void __launch_bounds__(kThreads, 1) select_tc_kernel(SelParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int kp = P.kp, t = P.t, ntiles = P.tiles;
  const uint32_t sbo = (uint32_t)kp * 32u;             // bytes between 8-row groups
  const uint32_t a_bytes = (uint32_t)kM * kp * 4u;     // one part (hi or lo) of the queries
  const uint32_t b_part = (uint32_t)kN * kp * 4u;      // one part of a codebook tile
  const uint32_t b_bytes = 2u * b_part;
  float* sA = reinterpret_cast<float*>(base);                        // hi, then lo at + a_bytes
  float* sB = reinterpret_cast<float*>(base + 2 * a_bytes);          // kStages x (hi, lo)
  float* park = reinterpret_cast<float*>(base + 2 * a_bytes + kStages * b_bytes);  // [kChunk][kM]
  uint64_t* bars = reinterpret_cast<uint64_t*>(park + kChunk * kM);  // full[2], empty[2], tfull[2], tempty[2]
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  __shared__ int issued_s, consumed_s, committed_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int s) { return tc::smem_u32(&bars[s]); };
  auto empty = [&](int s) { return tc::smem_u32(&bars[kStages + s]); };
  auto tfull = [&](int b) { return tc::smem_u32(&bars[2 * kStages + b]); };
  auto tempty = [&](int b) { return tc::smem_u32(&bars[2 * kStages + 2 + b]); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::bar_init(full(s), 1);
      tc::bar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::bar_init(tfull(b), 1);
      tc::bar_init(tempty(b), 4);
    }
    tc::bar_init_fence();
    abort_s = 0;
    issued_s = consumed_s = committed_s = 0;
  }
  if (warp == 1) tc::tmem_alloc(tc::smem_u32(&tmem_base_s), 2 * kN);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base_s;
  volatile int* abort_v = &abort_s;
  auto give_up = [&]() {
    if (atomicExch(&abort_s, 1) == 0) atomicExch(P.err, 1);
  };
  const int64_t q0 = (int64_t)blockIdx.x * kM;
  const int nqb = (int)min((int64_t)kM, P.nq - q0);
  const int m = 32 * (warp & 3) + lane;   // epilogue: query slot = TMEM lane

  // ---- queries -> hi / lo A operands (rows past the batch are zero); the
  // row's loads go out 16 at a time so that their latencies overlap
  if (warp >= 3) {
    const float* q = P.Qf + (q0 + m) * (int64_t)P.qstride;
    const int64_t row = (int64_t)(m >> 3) * (8 * kp) + (m & 7) * 4;
    constexpr int kBatch = 16;
    for (int b0 = 0; b0 < kp / 4; b0 += kBatch) {
      float4 v[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int k4 = b0 + u;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m < nqb && k4 < kp / 4 && 4 * k4 < P.qstride) v[u] = *reinterpret_cast<const float4*>(q + 4 * k4);
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int k4 = b0 + u;
        if (k4 >= kp / 4) break;
        const float e[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
        float h[4], l[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const float x = 4 * k4 + w < P.d ? e[w] : 0.f;
          h[w] = round_tf32(x);
          l[w] = round_tf32(x - h[w]);
        }
        *reinterpret_cast<float4*>(sA + row + k4 * 32) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(sA + a_bytes / 4 + row + k4 * 32) = make_float4(l[0], l[1], l[2], l[3]);
      }
    }
    tc::fence_async_smem();
  }
  if (warp > 0) asm volatile("bar.sync 3, %0;" ::"n"(kThreads - 32) : "memory");

  if (warp == 0) {
    // ---- producer: one bulk copy per codebook tile (hi and lo together)
    if (lane == 0) {
      for (int i = 0; i < ntiles; ++i) {
        const uint32_t s = i % kStages, ph = (i / kStages) & 1;
        if (!tc::bar_wait(empty(s), ph ^ 1, abort_v)) { give_up(); break; }
        tc::bar_arrive_expect_tx(full(s), b_bytes);
        tc::bulk_copy_g2s(tc::smem_u32(sB) + s * b_bytes, P.cb + (int64_t)i * (b_bytes / 4), b_bytes, full(s));
        issued_s = i + 1;
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: three tf32 passes per tile into TMEM buffer i % 2
    const uint32_t idesc = tc::idesc_tf32(kM, kN);
    int committed = 0;
    for (int i = 0; i < ntiles; ++i) {
      if (tc::named_bar_or(2, 64, false)) break;
      const uint32_t s = i % kStages, b = i & 1;
      if (lane == 0) {
        tc::fence_after_sync();
        const uint32_t ahi = tc::smem_u32(sA), alo = ahi + a_bytes;
        const uint32_t bhi = tc::smem_u32(sB) + s * b_bytes, blo = bhi + b_part;
        const uint32_t d = tmem + b * kN;
        for (int j = 0; j < kp / 8; ++j)
          tc::mma_tf32(d, tc::smem_desc(ahi + j * 256, 128, sbo), tc::smem_desc(bhi + j * 256, 128, sbo), idesc, j > 0);
        for (int j = 0; j < kp / 8; ++j)
          tc::mma_tf32(d, tc::smem_desc(ahi + j * 256, 128, sbo), tc::smem_desc(blo + j * 256, 128, sbo), idesc, 1);
        for (int j = 0; j < kp / 8; ++j)
          tc::mma_tf32(d, tc::smem_desc(alo + j * 256, 128, sbo), tc::smem_desc(bhi + j * 256, 128, sbo), idesc, 1);
        tc::mma_commit(empty(s));                   // the stage is free once these MMAs completed
        tc::mma_commit(tfull(b));
      }
      __syncwarp();
      committed = i + 1;
    }
    if (lane == 0) committed_s = committed;
  } else if (warp == 2) {
    // ---- gate: waits for each tile's stage and TMEM buffer, then releases
    // the MMA issuer
    for (int i = 0; i < ntiles; ++i) {
      const uint32_t s = i % kStages, ph = (i / kStages) & 1, b = i & 1, tph = (i >> 1) & 1;
      int ok = 1;
      if (lane == 0) {
        ok = tc::bar_wait(full(s), ph, abort_v) && tc::bar_wait(tempty(b), tph ^ 1, abort_v);
        if (!ok) give_up();
        else consumed_s = i + 1;
        tc::fence_before_sync();
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (tc::named_bar_or(2, 64, !ok)) break;
    }
  } else {
    // ---- epilogue: the query's t best (score, centroid id) in the last t
    // of TMAX slots, best first; the first TMAX - t slots hold +inf, which no
    // insertion passes, so the t-th best always sits in the last slot (a
    // fixed register)
    const bool active = m < nqb;
    const int lead = TMAX - t;
    float ts[TMAX];
    int ti[TMAX];
#pragma unroll
    for (int j = 0; j < TMAX; ++j) { ts[j] = j < lead ? INFINITY : -INFINITY; ti[j] = -1; }
    float cut = -INFINITY;                           // the t-th best score (-inf until t are held)
    for (int i = 0; i < ntiles; ++i) {
      const uint32_t b = i & 1, tph = (i >> 1) & 1;
      const bool ok = tc::bar_wait(tfull(b), tph, abort_v);
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
      const int col0 = i * kN;
      const int nvalid = min(kN, P.c - col0);
#pragma unroll
      for (int ch = 0; ch < kN / kChunk; ++ch) {
        // screen 16 columns against the cut (+inf for an idle slot; columns
        // past c are cleared afterwards); survivors parked in smem
        const float cut0 = active ? cut : INFINITY;
        uint32_t mk0 = 0, mk1 = 0;
#pragma unroll
        for (int cc = 0; cc < kChunk; ++cc) {
          const int c = ch * kChunk + cc;
          const float v = __uint_as_float(c < 32 ? r0[c & 31] : r1[c & 31]);
          if (v > cut0) {
            if (cc < kChunk / 2) mk0 |= 1u << cc;
            else mk1 |= 1u << cc;
            park[cc * kM + m] = v;
          }
        }
        uint32_t mask = mk0 | mk1;
        if (nvalid < kN) mask &= ch * kChunk >= nvalid ? 0u : nvalid - ch * kChunk >= 32 ? ~0u : (1u << (nvalid - ch * kChunk)) - 1;
        for (; mask; mask &= mask - 1) {
          const int cc = __ffs(mask) - 1;
          float v = park[cc * kM + m];
          if (!(v > cut)) continue;
          int id = col0 + ch * kChunk + cc;
#pragma unroll
          for (int j = 0; j < TMAX; ++j) {
            const bool gt = v > ts[j];
            const float tv = ts[j];
            const int tid = ti[j];
            ts[j] = gt ? v : tv;
            ti[j] = gt ? id : tid;
            v = gt ? tv : v;
            id = gt ? tid : id;
          }
          cut = ts[TMAX - 1];
        }
      }
    }
    if (active && !abort_s) {
      const int64_t q = q0 + m;
#pragma unroll
      for (int j = 0; j < TMAX; ++j) {
        if (j >= lead) {
          // an entry stays empty only when fewer than t scores exceed -inf
          // (NaN or -inf rows):
          // keep the ids valid partitions all the same
          P.top[q * t + j - lead] = ti[j] >= 0 ? ti[j] : j - lead;
          if (P.top_s) P.top_s[q * t + j - lead] = ts[j];
        }
      }
    }
  }

  // ---- teardown: after an abort, let copies and MMAs in flight land first
  __syncthreads();
  if (abort_s && threadIdx.x == 0) {
    volatile int never = 0;
    for (int i = consumed_s; i < issued_s; ++i) tc::bar_wait(full(i % kStages), (i / kStages) & 1, &never);
  }
  if (abort_s && threadIdx.x == 64 && committed_s > 0) {
    volatile int never = 0;
    const int i = committed_s - 1;
    tc::bar_wait(tfull(i & 1), (i >> 1) & 1, &never);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, 2 * kN);
}

size_t select_smem_bytes(int kp) {
  return 1024 + 2 * (size_t)kM * kp * 4 + kStages * 2 * (size_t)kN * kp * 4 + (size_t)kChunk * kM * 4 +
         (size_t)(2 * kStages + 4) * 8;
}

}  // namespace

bool select_tc_fits(int kp) { return kp % 8 == 0 && select_smem_bytes(kp) <= 227 * 1024 - 1024; }

void pack_select_codebook(const IndexData& ix, float* out, cudaStream_t s) {
  const int64_t total = (int64_t)ix.sel_tiles * kN * ix.sel_kp;
  pack_codebook_split<<<ceil_div(total, 256), 256, 0, s>>>(ix.centroids, ix.c, ix.d, ix.sel_kp, ix.sel_tiles, out);
  SOAR_LAUNCHED();
}

bool select_tc_usable(const IndexData& ix, const float* Qf, int qstride, int t) {
  return ix.sel_cb != nullptr && t >= 1 && t <= 32 && qstride % 4 == 0 &&
         (reinterpret_cast<uintptr_t>(Qf) & 15u) == 0;
}

void select_tc(const IndexData& ix, const float* Qf, int64_t nq, int qstride, int t, int32_t* top, float* top_s,
               cudaStream_t s) {
  SOAR_REQUIRE(select_tc_usable(ix, Qf, qstride, t), "tensor-core selection not applicable");
  if (nq == 0) return;
  SelParams P{Qf, nq, qstride, ix.d, ix.sel_kp, ix.sel_cb, ix.c, ix.sel_tiles, t, top, top_s, device_error_word()};
  const size_t smem = select_smem_bytes(ix.sel_kp);
  auto kern = t <= 16 ? select_tc_kernel<16> : select_tc_kernel<32>;
  SOAR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<ceil_div(nq, kM), kThreads, smem, s>>>(P);
  SOAR_LAUNCHED();
}

}  // namespace soar
