// Query-major exact IVF scan (Section 2.2 search, Section 3.5 deduplication)
// for batches whose probes spread thin over the partitions.
//
// The tensor-core scan (scan_tc.cu) streams each probed partition once and
// scores it against every query that probes it, 128 query slots per work
// item.  When a partition is probed by about one query (many partitions, few
// queries: two-level selection over 10^5 partitions, or a small serving
// batch), those items run almost empty and the scan is bound by per-tile
// epilogue work instead of HBM.  Here a warp takes one (query, probe) pair
// and walks that partition in the index's core-matrix copy of the rows:
// lane l scores row l of each 32-row block (four 8-row groups, so one
// 16-byte load per lane covers four whole 128-byte lines), the exact fp32
// dot product of the stored row with the query (elements in ascending order,
// the query in shared memory), and the warp keeps the pair's k best (score,
// id) rank keys, lane j the j-th.  Each pair's list is written best first;
// the caller's k-way merge over a query's lists drops the second copy of a
// spilled point (its exact score and id are identical).  Every probed pair
// reads its rows once; a warp per pair keeps the whole GPU busy even for a
// batch of a few queries.
#include "internal.cuh"
#include "scan_common.cuh"

namespace soar {

namespace {

constexpr int kQmWarps = 8;        // queries per block
constexpr int kQmMaxKp = 1024;     // query row (fp32) in shared memory: kQmWarps * kp * 4 bytes

// One 16-byte chunk of a stored row against the matching query elements.
template <typename T> struct Chunk;
template <> struct Chunk<float> {
  static constexpr int E = 4;
  __device__ static float dot(const uint4 w, const float* __restrict__ q, float acc) {
    const float4 a = *reinterpret_cast<const float4*>(q);
    acc = fmaf(a.x, __uint_as_float(w.x), acc);
    acc = fmaf(a.y, __uint_as_float(w.y), acc);
    acc = fmaf(a.z, __uint_as_float(w.z), acc);
    acc = fmaf(a.w, __uint_as_float(w.w), acc);
    return acc;
  }
};
template <> struct Chunk<__nv_bfloat16> {
  static constexpr int E = 8;
  // bf16 -> fp32 is exact: the 16 bits become the high half of the fp32 word
  __device__ static float dot(const uint4 w, const float* __restrict__ q, float acc) {
    const float4 a0 = *reinterpret_cast<const float4*>(q);
    const float4 a1 = *reinterpret_cast<const float4*>(q + 4);
    acc = fmaf(a0.x, __uint_as_float(w.x << 16), acc);
    acc = fmaf(a0.y, __uint_as_float(w.x & 0xffff0000u), acc);
    acc = fmaf(a0.z, __uint_as_float(w.y << 16), acc);
    acc = fmaf(a0.w, __uint_as_float(w.y & 0xffff0000u), acc);
    acc = fmaf(a1.x, __uint_as_float(w.z << 16), acc);
    acc = fmaf(a1.y, __uint_as_float(w.z & 0xffff0000u), acc);
    acc = fmaf(a1.z, __uint_as_float(w.w << 16), acc);
    acc = fmaf(a1.w, __uint_as_float(w.w & 0xffff0000u), acc);
    return acc;
  }
};

template <typename T>
__global__ void __launch_bounds__(32 * kQmWarps) scan_by_query_kernel(
    const T* __restrict__ rows, int kp, const int32_t* __restrict__ row_ids, const int64_t* __restrict__ gstart,
    const float* __restrict__ Qf, int qstride, const int32_t* __restrict__ top, const int32_t* __restrict__ tpq,
    int64_t nq, int t, int k, Cand* __restrict__ lists) {
  constexpr unsigned kFull = 0xffffffffu;
  constexpr int E = Chunk<T>::E;
  extern __shared__ __align__(16) float q_all[];   // [kQmWarps][kp]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * kQmWarps + w;   // pair q * t + j
  if (e >= nq * t) return;                                // uniform within the warp
  const int64_t q = e / t;
  const int j = (int)(e - q * t);
  Cand* out = lists + e * k;
  const int tq = tpq ? min(max(tpq[q], 0), t) : t;
  if (j >= tq) {                                          // probe not taken: an empty list
    if (lane < k) out[lane] = Cand{-INFINITY, -1};
    return;
  }
  float* qs = q_all + w * kp;
  for (int i = lane; i < kp; i += 32) qs[i] = Qf[q * (int64_t)qstride + i];
  __syncwarp();
  uint64_t mine = ~0ull;          // lane j < k: the j-th best key so far (empty: after every real key)
  uint64_t thr = ~0ull;           // the k-th best key
  const int chunks = kp / E;
  const size_t group_bytes = (size_t)8 * kp * sizeof(T);
  const unsigned char* base = reinterpret_cast<const unsigned char*>(rows) + (lane & 7) * 16;
  const int p = top[e];
  const int64_t g1 = gstart[p + 1];
  for (int64_t g = gstart[p]; g < g1; g += 4) {
    const int64_t gl = g + (lane >> 3);
    uint64_t key = ~0ull;
    if (gl < g1) {
      const int32_t id = row_ids[gl * 8 + (lane & 7)];
      if (id >= 0) {                                // -1: padding row of the group
        const unsigned char* x = base + gl * group_bytes;
        float acc = 0.f;
#pragma unroll 8
        for (int c = 0; c < chunks; ++c)
          acc = Chunk<T>::dot(__ldg(reinterpret_cast<const uint4*>(x + c * 128)), qs + c * E, acc);
        key = rank_key(acc, (uint32_t)id);
      }
    }
    // the 32 keys of this block into the warp's top k, one at a time
    unsigned bal = __ballot_sync(kFull, key < thr);
    while (bal) {
      const int src = __ffs(bal) - 1;
      bal &= bal - 1;
      const uint64_t kk = __shfl_sync(kFull, key, src);
      if (kk >= thr) continue;                                   // the same in every lane
      const int pos = __popc(__ballot_sync(kFull, lane < k && mine < kk));
      const uint64_t up = __shfl_up_sync(kFull, mine, 1);
      if (lane > pos && lane < k) mine = up;
      if (lane == pos) mine = kk;
      thr = __shfl_sync(kFull, mine, k - 1);
    }
  }
  if (lane < k) {
    const bool have = mine != ~0ull;
    out[lane] = have ? Cand{key_float(~(uint32_t)(mine >> 32)), (int32_t)(uint32_t)(mine & 0xffffffffu)}
                     : Cand{-INFINITY, -1};
  }
}

}  // namespace

bool scan_by_query_usable(const IndexData& ix, int64_t nq, int t, int k) {
  // thin probes: at most two (query, partition) pairs per partition on average
  return ix.tc_rows && ix.mode == SOAR_SCORE_F32 && k <= 32 && ix.tc_kp <= kQmMaxKp &&
         nq * (int64_t)t <= 2 * (int64_t)ix.c;
}

void scan_by_query(const IndexData& ix, const float* Qf, int qstride, const int32_t* top, const int32_t* tpq,
                   int64_t nq, int t, int k, Cand* lists, cudaStream_t s) {
  const size_t smem = (size_t)kQmWarps * ix.tc_kp * sizeof(float);
  const unsigned grid = ceil_div(nq * t, kQmWarps);
  if (ix.dtype == SOAR_F32)
    scan_by_query_kernel<float><<<grid, 32 * kQmWarps, smem, s>>>(
        static_cast<const float*>(ix.tc_rows), ix.tc_kp, ix.tc_ids, ix.tc_gstart, Qf, qstride, top, tpq, nq, t, k,
        lists);
  else
    scan_by_query_kernel<__nv_bfloat16><<<grid, 32 * kQmWarps, smem, s>>>(
        static_cast<const __nv_bfloat16*>(ix.tc_rows), ix.tc_kp, ix.tc_ids, ix.tc_gstart, Qf, qstride, top, tpq,
        nq, t, k, lists);
  SOAR_LAUNCHED();
}

}  // namespace soar
