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
// the query in shared memory), two rows per lane in flight, and the warp
// keeps the pair's 32 best (score, id) rank keys, lane j the j-th: a block
// with many newcomers is sorted across the warp and merged (bitonic), a
// block with few is inserted key by key.  Each pair's list is written best first;
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

// Ascending sort of one 64-bit key per lane across the warp (bitonic network).
__device__ __forceinline__ uint64_t warp_sort_keys(uint64_t v, int lane) {
#pragma unroll
  for (int kk = 2; kk <= 32; kk <<= 1)
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, v, j);
      const bool keep_min = ((lane & j) == 0) == ((lane & kk) == 0);
      v = keep_min ? (o < v ? o : v) : (o > v ? o : v);
    }
  return v;
}

// The warp's running 32 smallest keys (lane j: the j-th, ascending) merged
// with a block of 32 keys, one per lane.
__device__ __forceinline__ uint64_t merge_block(uint64_t mine, uint64_t key, uint64_t thr, int lane) {
  constexpr unsigned kFull = 0xffffffffu;
  unsigned bal = __ballot_sync(kFull, key < thr);
  if (__popc(bal) >= 4) {
    // many newcomers: sort the block, take the lane-wise minimum of the list
    // and the reversed block (a bitonic sequence holding the 32 smallest of
    // both), then sort that sequence
    const uint64_t b = warp_sort_keys(key, lane);
    const uint64_t r = __shfl_sync(kFull, b, 31 - lane);
    uint64_t c = r < mine ? r : mine;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
      const uint64_t o = __shfl_xor_sync(kFull, c, j);
      c = (lane & j) == 0 ? (o < c ? o : c) : (o > c ? o : c);
    }
    return c;
  }
  // a few newcomers: insert them one at a time
  uint64_t t31 = thr;
  while (bal) {
    const int src = __ffs(bal) - 1;
    bal &= bal - 1;
    const uint64_t kk = __shfl_sync(kFull, key, src);
    if (kk >= t31) continue;
    const int pos = __popc(__ballot_sync(kFull, mine < kk));
    const uint64_t up = __shfl_up_sync(kFull, mine, 1);
    if (lane > pos) mine = up;
    if (lane == pos) mine = kk;
    t31 = __shfl_sync(kFull, mine, 31);
  }
  return mine;
}

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
  const int p = top[e];
  float* qs = q_all + w * kp;
  for (int i = lane; i < kp; i += 32) qs[i] = Qf[q * (int64_t)qstride + i];
  __syncwarp();
  // the 32 best keys so far, lane j the j-th (~0: empty); the list keeps 32
  // entries whatever k, and its first k are the pair's top k
  uint64_t mine = ~0ull;
  const int chunks = kp / E;
  const size_t group_bytes = (size_t)8 * kp * sizeof(T);
  const unsigned char* base = reinterpret_cast<const unsigned char*>(rows) + (lane & 7) * 16;
  const int64_t g1 = gstart[p + 1];
  // two 32-row blocks per iteration (lane l: row l of each), so that each
  // lane has two rows' loads in flight
  for (int64_t g = gstart[p]; g < g1; g += 8) {
    const int64_t ga = g + (lane >> 3), gb = ga + 4;
    const bool va = ga < g1, vb = gb < g1;
    const int32_t ida = va ? row_ids[ga * 8 + (lane & 7)] : -1;
    const int32_t idb = vb ? row_ids[gb * 8 + (lane & 7)] : -1;
    const unsigned char* xa = base + (va ? ga : 0) * group_bytes;
    const unsigned char* xb = base + (vb ? gb : 0) * group_bytes;
    float acc_a = 0.f, acc_b = 0.f;
#pragma unroll 2
    for (int c = 0; c < chunks; ++c) {
      const uint4 wa = __ldg(reinterpret_cast<const uint4*>(xa + c * 128));
      const uint4 wb = __ldg(reinterpret_cast<const uint4*>(xb + c * 128));
      acc_a = Chunk<T>::dot(wa, qs + c * E, acc_a);
      acc_b = Chunk<T>::dot(wb, qs + c * E, acc_b);
    }
    const uint64_t ka = ida >= 0 ? rank_key(acc_a, (uint32_t)ida) : ~0ull;   // -1: padding row or past the end
    const uint64_t kb = idb >= 0 ? rank_key(acc_b, (uint32_t)idb) : ~0ull;
    mine = merge_block(mine, ka, __shfl_sync(kFull, mine, 31), lane);
    mine = merge_block(mine, kb, __shfl_sync(kFull, mine, 31), lane);
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
