// Exact top-R shortlist of approximately scored candidates over each query's
// probed union (Section 3.5: compressed representations are duplicated for
// every assignment, the high-bitrate rows are stored once and rescore the
// best candidates), for two compressed layouts: per-row scaled E4M3 codes
// of every copy (approximate score s_q * s_x * sum q8 x8), and 4-bit PQ
// codes of every copy's residual x - C_p (approximate score <q, C_p> +
// sum_s <q_s, B[s][code_s]>).
//
// Three kernels:
//   pair_offsets  each probed pair's place in its query's slice of a key
//                 buffer (the sizes of the earlier probed partitions);
//   approx_pairs  a warp per (query, probe) pair scores the partition's rows
//                 (lane = row, code rows read coalesced), drops a copy when
//                 the point has another copy in a partition the query probed
//                 earlier (from the index's copy of the assignment: each
//                 point counts once) and writes one 64-bit rank key per row
//                 (approximate score descending, then id ascending; the
//                 all-ones key for a dropped copy);
//   select_top_r  a warp per query finds the R smallest keys of its slice by an MSB-first
//                 radix select over bytes (warp histograms in shared memory;
//                 the keys are distinct, so the selected set is exact) and
//                 writes their ids.
// The caller rescores those ids exactly from the stored rows.
#include "internal.cuh"
#include "scan_common.cuh"

namespace soar {

namespace {

constexpr int kSlWarps = 8;
constexpr int kSlMaxProbesSmem = 256;   // probe lists held in shared memory up to this t

__device__ __forceinline__ float fp8_code_value(uint32_t b) {
  __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
  return __half2float(__half(h));
}

// FP8 rows: approx = s_q * s_x * sum q8 x8 (products summed in fp32 in
// ascending element order); per warp the query's code values.
struct Fp8Rows {
  const uint8_t* codes;
  int code_stride;
  const float* row_scales;
  const float* Qf;        // [nq][code_stride] code values
  const float* qscale;
  __host__ __device__ int smem_floats() const { return code_stride; }
  __device__ void load(float* qs, int64_t q, int lane) const {
    for (int i = lane; i < code_stride; i += 32) qs[i] = Qf[q * (int64_t)code_stride + i];
  }
  __device__ float partition_base(const float*, int, int) const { return 0.f; }
  __device__ float score(const float* qs, int64_t q, int64_t r, float) const {
    const uint4* x = reinterpret_cast<const uint4*>(codes + r * (int64_t)code_stride);
    float acc = 0.f;
    for (int c = 0; c < code_stride / 16; ++c) {
      const uint4 v = __ldg(x + c);
      const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc = fmaf(qs[16 * c + 4 * i + b], fp8_code_value((wv[i] >> (8 * b)) & 0xffu), acc);
    }
    return acc * qscale[q] * row_scales[r];
  }
};

// PQ4 rows: approx = <q, C_p> + sum_s LUT[s][code_s] with LUT[s][j] =
// <q_s, B[s][j]>; per warp the LUT ([m][16]) followed by the query row.
struct Pq4Rows {
  const uint8_t* codes;
  int code_stride, m, d;
  const float* B;         // [m][16][2]
  const float* C;         // [c][d]
  const float* Qf;        // [nq][qstride] fp32
  int qstride;
  __host__ __device__ int smem_floats() const { return m * 16 + qstride; }
  __device__ void load(float* qs, int64_t q, int lane) const {
    float* qrow = qs + m * 16;
    for (int i = lane; i < qstride; i += 32) qrow[i] = Qf[q * (int64_t)qstride + i];
    for (int e = lane; e < m * 16; e += 32) {
      const int sidx = e / 16;
      const float q0 = Qf[q * (int64_t)qstride + 2 * sidx], q1 = Qf[q * (int64_t)qstride + 2 * sidx + 1];
      qs[e] = fmaf(q1, B[2 * e + 1], q0 * B[2 * e]);
    }
  }
  // <q, C_p> in fp32 (lanes over the dimensions, a fixed shuffle tree, lane 0's value to all)
  __device__ float partition_base(const float* qs, int p, int lane) const {
    const float* qrow = qs + m * 16;
    const float* cp = C + (int64_t)p * d;
    float v = 0.f;
    for (int k = lane; k < d; k += 32) v = fmaf(qrow[k], cp[k], v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
  }
  __device__ float score(const float* qs, int64_t, int64_t r, float base) const {
    const uint4* x = reinterpret_cast<const uint4*>(codes + r * (int64_t)code_stride);
    float acc = 0.f;
    for (int c = 0; c < code_stride / 16; ++c) {
      const uint4 v = __ldg(x + c);
      const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int sidx = 32 * c + 8 * i + b;        // nibble b of word i of chunk c
          if (sidx < m) acc += qs[16 * sidx + ((wv[i] >> (4 * b)) & 0xfu)];
        }
    }
    return base + acc;
  }
};

// Each probed pair's first position in its query's key slice: the sizes of
// the query's earlier probed partitions added up (a thread per query).
__global__ void pair_offsets(const int64_t* __restrict__ off, const int32_t* __restrict__ top,
                             const int32_t* __restrict__ tpq, int64_t q0, int64_t nq, int t,
                             int64_t* __restrict__ pos, int64_t* __restrict__ counts) {
  const int64_t ql = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ql >= nq) return;
  const int64_t q = q0 + ql;
  const int tq = tpq ? min(max(tpq[q], 0), t) : t;
  int64_t acc = 0;
  for (int j = 0; j < tq; ++j) {
    pos[ql * t + j] = acc;
    const int p = top[q * (int64_t)t + j];
    acc += off[p + 1] - off[p];
  }
  counts[ql] = acc;
}

// A warp per (query, probe) pair: the approximate score of every row of the
// probed partition, written as a rank key at the pair's place in the query's
// slice; a copy whose point has another copy in a partition the query probed
// earlier writes the all-ones key instead (it sorts after every real key and
// its id bits read as -1).
template <typename Rows>
__global__ void __launch_bounds__(32 * kSlWarps) approx_pairs(
    Rows rows, const int32_t* __restrict__ ids, const int64_t* __restrict__ off, const int32_t* __restrict__ assign,
    int a, const int32_t* __restrict__ top, const int32_t* __restrict__ tpq, int64_t q0, int64_t nq, int t,
    int64_t slice, const int64_t* __restrict__ pos, uint64_t* __restrict__ keys) {
  extern __shared__ __align__(16) unsigned char sl_smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t el = (int64_t)blockIdx.x * kSlWarps + w;   // pair within this chunk: ql * t + j
  if (el >= nq * t) return;                               // uniform within the warp
  const int64_t ql = el / t;
  const int j = (int)(el - ql * t);
  const int64_t q = q0 + ql;
  const int tq = tpq ? min(max(tpq[q], 0), t) : t;
  if (j >= tq) return;
  const int per = rows.smem_floats();
  float* qs = reinterpret_cast<float*>(sl_smem) + w * per;
  int32_t* probes_s = reinterpret_cast<int32_t*>(reinterpret_cast<float*>(sl_smem) + kSlWarps * per) +
                      w * kSlMaxProbesSmem;
  rows.load(qs, q, lane);
  const int32_t* probes = top + q * (int64_t)t;
  if (j <= kSlMaxProbesSmem) {
    for (int jj = lane; jj < j; jj += 32) probes_s[jj] = probes[jj];
    probes = probes_s;
  }
  __syncwarp();
  const int p = top[q * (int64_t)t + j];
  const float base = rows.partition_base(qs, p, lane);
  const int64_t r0 = off[p], r1 = off[p + 1];
  uint64_t* out = keys + ql * slice + pos[el] - r0;
  for (int64_t r = r0 + lane; r < r1; r += 32) {
    const int32_t id = ids[r];
    bool keep = true;
    // the point's copy in an earlier-probed partition is the one that counts
    for (int i = 0; i < a && keep; ++i) {
      const int other = assign[(int64_t)id * a + i];
      if (other == p) continue;
      for (int jj = 0; jj < j; ++jj)
        if (probes[jj] == other) { keep = false; break; }
    }
    out[r] = keep ? rank_key(rows.score(qs, q, r, base), (uint32_t)id) : ~0ull;
  }
}

// The R smallest keys of each query's slice -> their ids (cand [nq][R],
// padded with -1 when the slice holds fewer than R keys).
__global__ void __launch_bounds__(32 * kSlWarps) select_top_r(const uint64_t* __restrict__ keys,
                                                              const int64_t* __restrict__ counts, int64_t nq,
                                                              int64_t slice, int R, int32_t* __restrict__ cand) {
  constexpr unsigned kFull = 0xffffffffu;
  __shared__ int hist_all[kSlWarps][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t ql = (int64_t)blockIdx.x * kSlWarps + w;
  if (ql >= nq) return;
  const uint64_t* K = keys + ql * slice;
  const int64_t n = counts[ql];
  int32_t* out = cand + ql * (int64_t)R;
  int* hist = hist_all[w];
  uint64_t limit = ~0ull;                 // keys <= limit are selected
  if (n > R) {
    uint64_t prefix = 0, mask = 0;
    int64_t need = R;
    for (int shift = 56; shift >= 0; shift -= 8) {
      for (int b = lane; b < 256; b += 32) hist[b] = 0;
      __syncwarp();
      for (int64_t i = lane; i < n; i += 32) {
        const uint64_t kk = K[i];
        if ((kk & mask) == prefix) atomicAdd(&hist[(kk >> shift) & 0xff], 1);
      }
      __syncwarp();
      // lane l owns bins 8l .. 8l+7; a warp scan of their sums finds the
      // first bin whose inclusive count reaches `need`
      int v[8], s = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) { v[i] = hist[8 * lane + i]; s += v[i]; }
      int incl = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const int excl = incl - s;
      const unsigned hit = __ballot_sync(kFull, incl >= need);
      const int owner = __ffs(hit) - 1;           // need <= total, so some lane hits
      int bin = 0, before = 0, in_bin = 0;
      if (lane == owner) {
        int c = excl;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (c + v[i] >= need) { bin = 8 * lane + i; before = c; in_bin = v[i]; break; }
          c += v[i];
        }
      }
      bin = __shfl_sync(kFull, bin, owner);
      before = __shfl_sync(kFull, before, owner);
      in_bin = __shfl_sync(kFull, in_bin, owner);
      prefix |= (uint64_t)bin << shift;
      mask |= (uint64_t)0xff << shift;
      if (before + in_bin == need || shift == 0) {   // the whole bin fits: done
        limit = prefix | (shift ? (((uint64_t)1 << shift) - 1) : 0);
        break;
      }
      need -= before;
      __syncwarp();
    }
  }
  // every key below the limit, then keys equal to it (at most one real key:
  // the keys are distinct) until R are taken; a dropped copy's all-ones key
  // is never a real candidate, so the rest is padding
  int64_t m = 0;
  for (int pass = 0; pass < 2 && m < R; ++pass) {
    if (pass == 1 && limit == ~0ull) break;
    for (int64_t i0 = 0; i0 < n && m < R; i0 += 32) {
      const int64_t i = i0 + lane;
      const uint64_t kk = i < n ? K[i] : ~0ull;
      const bool take = i < n && (pass == 0 ? kk < limit : kk == limit);
      const unsigned bal = __ballot_sync(kFull, take);
      const int64_t pos = m + __popc(bal & ((1u << lane) - 1u));
      if (take && pos < R) out[pos] = (int32_t)(kk & 0xffffffffu);
      m += __popc(bal);
    }
  }
  for (int64_t i = min(m, (int64_t)R) + lane; i < R; i += 32) out[i] = -1;
}


template <typename Rows>
void run_shortlist(const IndexData& ix, const Rows& rws, const int32_t* top, const int32_t* tpq, int64_t nq, int t,
                   int R, int32_t* cand, cudaStream_t s, Scratch& scr) {
  const int64_t slice = std::max<int64_t>(1, std::min<int64_t>((int64_t)t * ix.max_partition, ix.rows));
  // queries per pass so that the key buffer stays within 2 GB
  const int64_t chunk = std::max<int64_t>(kSlWarps, std::min<int64_t>(nq, ((int64_t)1 << 28) / slice));
  const int64_t cq = std::min(chunk, nq);
  uint64_t* keys = scr.get<uint64_t>((size_t)cq * slice);
  int64_t* counts = scr.get<int64_t>(cq);
  int64_t* pos = scr.get<int64_t>((size_t)cq * t);
  const size_t smem = (size_t)kSlWarps * rws.smem_floats() * sizeof(float) + (size_t)kSlWarps * kSlMaxProbesSmem * 4;
  SOAR_CUDA(cudaFuncSetAttribute(approx_pairs<Rows>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int a = 1 + ix.spills;
  for (int64_t q0 = 0; q0 < nq; q0 += cq) {
    const int64_t m = std::min(cq, nq - q0);
    pair_offsets<<<ceil_div(m, 128), 128, 0, s>>>(ix.offsets, top, tpq, q0, m, t, pos, counts);
    SOAR_LAUNCHED();
    approx_pairs<Rows><<<ceil_div(m * t, kSlWarps), 32 * kSlWarps, smem, s>>>(rws, ix.ids, ix.offsets, ix.assign, a,
                                                                              top, tpq, q0, m, t, slice, pos, keys);
    SOAR_LAUNCHED();
    select_top_r<<<ceil_div(m, kSlWarps), 32 * kSlWarps, 0, s>>>(keys, counts, m, slice, R, cand + q0 * R);
    SOAR_LAUNCHED();
  }
}

}  // namespace

void fp8_shortlist(const IndexData& ix, const float* Qf, const float* qscale, const int32_t* top,
                   const int32_t* tpq, int64_t nq, int t, int R, int32_t* cand, cudaStream_t s, Scratch& scr) {
  const Fp8Rows rws{static_cast<const uint8_t*>(ix.vectors), ix.code_stride, ix.row_scales, Qf, qscale};
  run_shortlist(ix, rws, top, tpq, nq, t, R, cand, s, scr);
}

void pq_shortlist(const IndexData& ix, const float* Qf, int qstride, const int32_t* top, const int32_t* tpq,
                  int64_t nq, int t, int R, int32_t* cand, cudaStream_t s, Scratch& scr) {
  const Pq4Rows rws{static_cast<const uint8_t*>(ix.vectors), ix.code_stride, ix.pq_m, ix.d, ix.pq_cb, ix.centroids,
                    Qf, qstride};
  run_shortlist(ix, rws, top, tpq, nq, t, R, cand, s, scr);
}

}  // namespace soar
