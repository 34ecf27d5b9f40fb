// Query side of the SOAR IVF index (Section 2.2, Section 3.5) and exact
// brute-force MIPS (Section 2.1).
//
//   prep     queries -> fp32 rows padded like the index rows (FP8 indices:
//            per-query scaled E4M3 code values + scale)
//   score    S = Q . C^T (tiled fp32 GEMM; FP8 indices scale the code product)
//   top-t    per query: 4-pass radix select of the t-th best key, compaction
//            (ties at the threshold go to the lower id), bitonic sort in smem
//   group    (query, probe) pairs sorted by partition (stable radix sort):
//            every partition is read once per batch for all its queries
//   scan     persistent CTAs take (partition, <=64 queries) work items,
//            biggest partitions first; a register-tiled dot product per
//            (query, row) and a per-query top-k list in shared memory
//   merge    warp per query: k-way merge of its per-partition lists by
//            (score desc, id asc); a spilled point scored in two partitions
//            has bit-identical (score, id) in both, so the copies are
//            adjacent and the second is dropped (deduplication, Section 3.5)
//   rescore  FP8 indices: the merged candidates are rescored exactly in fp32
//            from the single stored copy and the top k kept
#include <algorithm>

#include "internal.cuh"
#include "scan_common.cuh"

namespace soar {

namespace {

constexpr int QB = 64;          // query slots per work item
constexpr int RB = 64;          // rows per tile
constexpr int SSTRIDE = RB + 4; // score tile stride (conflict-free epilogue reads)
constexpr int kThreads = 256;

// smem row stride (floats) for a row of `row_stride` elements: >= row_stride,
// a multiple of 4, and == 4 (mod 32) so 8 consecutive rows read by float4
// land in distinct banks.
inline int smem_stride(int row_stride) {
  int xs = (row_stride + 3) / 4 * 4;
  while (xs % 32 != 4) xs += 4;
  return xs;
}

// ------------------------------------------------------------ row expansion

template <typename T> struct Expand;
template <> struct Expand<float> {
  static constexpr int kPer = 4;
  __device__ static void to(uint4 v, float* dst) {
    *reinterpret_cast<float4*>(dst) = make_float4(__uint_as_float(v.x), __uint_as_float(v.y),
                                                  __uint_as_float(v.z), __uint_as_float(v.w));
  }
};
template <> struct Expand<__nv_bfloat16> {
  static constexpr int kPer = 8;
  __device__ static void to(uint4 v, float* dst) {
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      dst[2 * i] = __uint_as_float(w[i] << 16);
      dst[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
};
__device__ __forceinline__ float fp8_value(uint8_t b) {
  __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
  return __half2float(__half(h));
}

// ------------------------------------------------------------ query prep

// Warp per query.  Plain: fp32 copy padded with zeros to `stride`.
// FP8: code values of e4m3(q / scale), scale = max|q| / 448.
// qnorm (optional): ||row|| of the written row.
template <typename QT>
__global__ void prep_queries(const QT* __restrict__ Q, int64_t nq, int d, int stride, bool fp8,
                             float* __restrict__ Qf, float* __restrict__ qscale, float* __restrict__ qnorm) {
  int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (q >= nq) return;
  const QT* src = Q + q * d;
  float* dst = Qf + q * stride;
  float scale = 1.f;
  if (fp8) {
    float amax = 0.f;
    for (int k = lane; k < d; k += 32) amax = fmaxf(amax, fabsf(load_elem(src, k)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    scale = amax > 0.f ? amax / 448.f : 1.f;
  }
  float acc = 0.f;
  for (int k = lane; k < stride; k += 32) {
    float v = k < d ? load_elem(src, k) : 0.f;
    if (fp8 && k < d)
      v = fp8_value((uint8_t)__nv_cvt_float_to_fp8(v / scale, __NV_SATFINITE, __NV_E4M3));
    dst[k] = v;
    acc = fmaf(v, v, acc);
  }
  if (fp8 && lane == 0) qscale[q] = scale;
  if (qnorm) {
    acc = warp_sum(acc);
    if (lane == 0) qnorm[q] = sqrtf(acc);
  }
}

// ------------------------------------------------------------ centroid scores

// S[q][i] = sum_k A[q][k] * B[i][k] (* ascale[q] * bscale[i] when given).
// A rows have stride lda, B rows stride ldb; both hold >= d valid columns.
__global__ void __launch_bounds__(256) gemm_nt(const float* __restrict__ A, int64_t m, int lda,
                                               const float* __restrict__ B, int nb, int ldb, int d,
                                               const float* __restrict__ ascale,
                                               const float* __restrict__ bscale, float* __restrict__ S) {
  constexpr int TBM = 64, TBN = 64, TBK = 16;
  __shared__ __align__(16) float As[TBK][TBM];
  __shared__ __align__(16) float Bs[TBK][TBN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * TBM;
  const int n0 = blockIdx.x * TBN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < d; k0 += TBK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int idx = tid + e * 256, r = idx / TBK, kk = idx % TBK, k = k0 + kk;
      As[kk][r] = (m0 + r < m && k < d) ? A[(m0 + r) * lda + k] : 0.f;
      Bs[kk][r] = (n0 + r < nb && k < d) ? B[(int64_t)(n0 + r) * ldb + k] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TBK; ++kk) {
      float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t r = m0 + ty * 4 + i;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int col = n0 + tx * 4 + j;
      if (col >= nb) continue;
      float v = acc[i][j];
      if (ascale) v = v * ascale[r] * bscale[col];
      S[r * nb + col] = v;
    }
  }
}

// Tiled fp32 GEMM S = A . B^T (same contract as gemm_nt) for 16-byte aligned
// rows: 128 x 128 block tile, 8 x 8 outputs per thread, K in steps of 8 with
// the next step prefetched into registers while the current one computes.
__global__ void __launch_bounds__(256) gemm_nt_128(const float* __restrict__ A, int64_t m, int lda,
                                                   const float* __restrict__ B, int nb, int ldb, int d,
                                                   const float* __restrict__ ascale,
                                                   const float* __restrict__ bscale, float* __restrict__ S) {
  constexpr int TB = 128, TK = 8;
  __shared__ __align__(16) float As[2][TK][TB];
  __shared__ __align__(16) float Bs[2][TK][TB];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * TB;
  const int n0 = blockIdx.x * TB;
  // loader: thread -> (row lr, k-quad lq) of a 128 x 8 tile, one float4 each for A and B
  const int lr = tid >> 1, lq = (tid & 1) * 4;
  const bool arow = m0 + lr < m, brow = n0 + lr < nb;
  const float* ap = A + (m0 + lr) * (int64_t)lda;
  const float* bp = B + (int64_t)(n0 + lr) * ldb;
  auto load = [&](int k0, float4& va, float4& vb) {
    const int k = k0 + lq;
    va = (arow && k < d) ? *reinterpret_cast<const float4*>(ap + k) : make_float4(0.f, 0.f, 0.f, 0.f);
    vb = (brow && k < d) ? *reinterpret_cast<const float4*>(bp + k) : make_float4(0.f, 0.f, 0.f, 0.f);
    // columns k+1..k+3 beyond d are zero in A's padded rows; B rows are read to
    // the next multiple of 4, so clear them explicitly
    if (k + 3 >= d) {
      if (k + 1 >= d) { va.y = 0.f; vb.y = 0.f; }
      if (k + 2 >= d) { va.z = 0.f; vb.z = 0.f; }
      if (k + 3 >= d) { va.w = 0.f; vb.w = 0.f; }
    }
  };
  auto store = [&](int buf, const float4& va, const float4& vb) {
    As[buf][lq + 0][lr] = va.x; As[buf][lq + 1][lr] = va.y; As[buf][lq + 2][lr] = va.z; As[buf][lq + 3][lr] = va.w;
    Bs[buf][lq + 0][lr] = vb.x; Bs[buf][lq + 1][lr] = vb.y; Bs[buf][lq + 2][lr] = vb.z; Bs[buf][lq + 3][lr] = vb.w;
  };
  float acc[8][8] = {};
  float4 va, vb;
  load(0, va, vb);
  store(0, va, vb);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < d; k0 += TK) {
    const bool more = k0 + TK < d;
    if (more) load(k0 + TK, va, vb);
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) {
      store(buf ^ 1, va, vb);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (col >= nb) continue;
      float v = acc[i][j];
      if (ascale) v = v * ascale[r] * bscale[col];
      S[r * nb + col] = v;
    }
  }
}

// ------------------------------------------------------------ top-t select

// One block per row of S: the t best columns (score desc, lower id on ties),
// sorted.  Dynamic smem: pow2 >= t 64-bit keys, then the row itself when
// c <= kToptSmemRow.
constexpr int kToptSmemRow = 12288;
__global__ void __launch_bounds__(256) topt_kernel(const float* __restrict__ S, int c, int t, int t2,
                                                   int32_t* __restrict__ top, float* __restrict__ top_s) {
  extern __shared__ uint64_t buf[];
  __shared__ int hist[256];
  __shared__ uint32_t prefix_s;
  __shared__ int remaining_s;
  __shared__ int gt_cnt, eq_base;
  __shared__ int warp_eq[8];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t q = blockIdx.x;
  const float* row = S + q * c;
  if (c <= kToptSmemRow) {
    // the row is read four times: keep it in shared memory behind the sort buffer
    float* srow = reinterpret_cast<float*>(buf + t2);
    for (int i = tid; i < c; i += 256) srow[i] = row[i];
    __syncthreads();
    row = srow;
  }
  uint32_t prefix = 0;
  int remaining = t;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    const uint32_t hmask = pass == 0 ? 0u : (0xffffffffu << (shift + 8));
    hist[tid] = 0;
    __syncthreads();
    for (int i = tid; i < c; i += 256) {
      uint32_t key = float_key(row[i]);
      if ((key & hmask) == (prefix & hmask)) atomicAdd(&hist[(key >> shift) & 255u], 1);
    }
    __syncthreads();
    if (tid == 0) {
      int acc = 0, D = 255;
      for (; D > 0; --D) {
        if (acc + hist[D] >= remaining) break;
        acc += hist[D];
      }
      remaining_s = remaining - acc;
      prefix_s = prefix | ((uint32_t)D << shift);
    }
    __syncthreads();
    prefix = prefix_s;
    remaining = remaining_s;
    __syncthreads();
  }
  const uint32_t T = prefix;
  if (tid == 0) { gt_cnt = 0; eq_base = 0; }
  __syncthreads();
  const int n_gt = t - remaining;
  for (int c0 = 0; c0 < c; c0 += 256) {
    int i = c0 + tid;
    uint32_t key = i < c ? float_key(row[i]) : 0u;
    bool gt = i < c && key > T;
    bool eq = i < c && key == T;
    if (gt) {
      int slot = atomicAdd(&gt_cnt, 1);
      buf[slot] = rank_key(row[i], (uint32_t)i);
    }
    unsigned bal = __ballot_sync(0xffffffffu, eq);
    if (lane == 0) warp_eq[w] = __popc(bal);
    __syncthreads();
    int before = eq_base;
    for (int ww = 0; ww < w; ++ww) before += warp_eq[ww];
    int rank = before + __popc(bal & ((1u << lane) - 1u));
    if (eq && rank < remaining) buf[n_gt + rank] = rank_key(row[i], (uint32_t)i);
    __syncthreads();
    if (tid == 0) {
      int s = 0;
      for (int ww = 0; ww < 8; ++ww) s += warp_eq[ww];
      eq_base += s;
    }
    __syncthreads();
  }
  for (int i = t + tid; i < t2; i += 256) buf[i] = ~0ull;
  __syncthreads();
  for (int size = 2; size <= t2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < t2; i += 256) {
        int j = i ^ stride;
        if (j > i) {
          bool up = (i & size) == 0;
          uint64_t a = buf[i], b = buf[j];
          if ((a > b) == up) { buf[i] = b; buf[j] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int j = tid; j < t; j += 256) {
    uint64_t key = buf[j];
    uint32_t id = (uint32_t)(key & 0xffffffffu);
    top[q * t + j] = (int32_t)id;
    if (top_s) top_s[q * t + j] = row[id];
  }
}

// Top-t for t <= 32, a warp per query: lane j holds the query's j-th best
// (score, id) key so far (ascending rank keys: higher score first, lower id
// on ties); the row streams through in coalesced chunks of 32, a ballot
// keeps the chunk's keys that beat the current t-th, and each is inserted by
// one ballot (its position) and one shuffle (the shift).
__global__ void __launch_bounds__(256) topt_warp_kernel(const float* __restrict__ S, int64_t nq, int c, int t,
                                                        int32_t* __restrict__ top, float* __restrict__ top_s) {
  constexpr unsigned kFull = 0xffffffffu;
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= nq) return;
  const float* row = S + q * c;
  uint64_t mine = ~0ull;          // empty entries rank after every real key
  uint64_t thr = ~0ull;           // the t-th best key
  // four chunks of 32 per step: their loads are issued together
  for (int c0 = 0; c0 < c; c0 += 128) {
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = c0 + 32 * u + lane;
      v[u] = i < c ? row[i] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = c0 + 32 * u + lane;
      const uint64_t key = i < c ? rank_key(v[u], (uint32_t)i) : ~0ull;
      unsigned bal = __ballot_sync(kFull, key < thr);
      while (bal) {
        const int src = __ffs(bal) - 1;
        bal &= bal - 1;
        const uint64_t kk = __shfl_sync(kFull, key, src);
        if (kk >= thr) continue;                     // the same in every lane
        const int pos = __popc(__ballot_sync(kFull, lane < t && mine < kk));
        const uint64_t up = __shfl_up_sync(kFull, mine, 1);
        if (lane > pos && lane < t) mine = up;
        if (lane == pos) mine = kk;
        thr = __shfl_sync(kFull, mine, t - 1);
      }
    }
  }
  if (lane < t) {
    const uint32_t id = (uint32_t)(mine & 0xffffffffu);
    top[q * t + lane] = (int32_t)id;
    if (top_s) top_s[q * t + lane] = row[id];
  }
}

// ------------------------------------------------------------ grouping

// top[q][j] = j: every query probes every partition (the flat index of the
// brute force).
__global__ void all_partitions(int32_t* __restrict__ top, int64_t nq, int c) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nq * c) top[e] = (int32_t)(e % c);
}

// Counting sort of the (query, probe) pairs by partition: per-partition
// counts (a probe beyond the query's own t counts in the sentinel bucket c),
// then a scatter that also records each pair's position (the inverse map).
// The order of the pairs inside a partition is immaterial to the search.
__global__ void pair_counts(const int32_t* __restrict__ top, int64_t nq, int tmax, const int32_t* __restrict__ tpq,
                            int c, unsigned long long* __restrict__ cnt, unsigned* __restrict__ first) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nq * tmax) return;
  const int64_t q = e / tmax;
  const int j = (int)(e - q * tmax);
  const int tq = tpq ? min(max(tpq[q], 0), tmax) : tmax;
  atomicAdd(&cnt[j < tq ? top[e] : c], 1ull);
  if (first && j == 0 && tq > 0) atomicAdd(&first[top[e]], 1u);
}

// The scan's partition order: the partitions that are the first probe of the
// most queries come first (their finished items publish those queries' bounds
// early), ties in the index's size order.  A counting rank in one launch: lane
// l of block b ranks partition size_order[32 b + l] against every other, the
// block's 8 warps splitting the comparisons; it costs less than a multi-pass
// radix sort's launches while c is small (c <= kRankMaxC).
constexpr int kRankTile = 4096;
constexpr int kRankMaxC = 16384;

__global__ void __launch_bounds__(256) first_probe_order(const int32_t* __restrict__ size_order,
                                                         const unsigned* __restrict__ first, int c,
                                                         int32_t* __restrict__ order) {
  __shared__ unsigned sk[kRankTile];
  __shared__ int rank_s[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  if (threadIdx.x < 32) rank_s[threadIdx.x] = 0;
  const unsigned ki = i < c ? first[size_order[i]] : 0u;
  int rank = 0;
  for (int j0 = 0; j0 < c; j0 += kRankTile) {
    const int m = min(kRankTile, c - j0);
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) sk[j] = first[size_order[j0 + j]];
    __syncthreads();
    for (int j = warp; j < m; j += 8) {
      const unsigned kj = sk[j];
      rank += (kj > ki) || (kj == ki && j0 + j < i);
    }
  }
  atomicAdd(&rank_s[lane], rank);
  __syncthreads();
  if (warp == 0 && i < c) order[rank_s[lane]] = size_order[i];
}

__global__ void pair_scatter(const int32_t* __restrict__ top, int64_t nq, int tmax, const int32_t* __restrict__ tpq,
                             int c, const int64_t* __restrict__ pair_off, int32_t* __restrict__ cursor,
                             int32_t* __restrict__ vals, int32_t* __restrict__ inv) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nq * tmax) return;
  const int64_t q = e / tmax;
  const int j = (int)(e - q * tmax);
  const int tq = tpq ? min(max(tpq[q], 0), tmax) : tmax;
  const int b = j < tq ? top[e] : c;
  const int64_t pos = pair_off[b] + atomicAdd(&cursor[b], 1);
  vals[pos] = (int32_t)e;
  inv[e] = (int32_t)pos;
}

// One block: the offsets of the grouped pairs and of the work items.
//   pair_off[0 .. c+2)  exclusive scan of the per-partition pair counts
//   item_base[0 .. c+1) exclusive scan of ceil(pairs / qb) over the
//                       partitions in `order` (the last entry: the total)
//   cursor[0 .. c+1)    zeroed for pair_scatter
// Each thread takes a run of consecutive entries, so one block scan covers
// any c.
constexpr int kOffThreads = 1024;
__global__ void __launch_bounds__(kOffThreads) group_offsets(const unsigned long long* __restrict__ cnt, int c,
                                                             const int32_t* __restrict__ order, int qb,
                                                             int64_t* __restrict__ pair_off,
                                                             int32_t* __restrict__ item_base,
                                                             int32_t* __restrict__ cursor) {
  __shared__ int64_t warp64[32];
  __shared__ int32_t warp32[32];
  const int tid = threadIdx.x;
  {
    const int n = c + 2, per = (n + kOffThreads - 1) / kOffThreads;
    const int i0 = min(n, tid * per), i1 = min(n, i0 + per);
    int64_t sum = 0;
    for (int i = i0; i < i1; ++i) sum += (int64_t)cnt[i];
    int64_t total;
    int64_t run = block_exclusive_scan<int64_t>(sum, warp64, total);
    for (int i = i0; i < i1; ++i) {
      pair_off[i] = run;
      run += (int64_t)cnt[i];
    }
  }
  __syncthreads();                       // pair_off complete and visible to the block
  {
    const int n = c + 1, per = (n + kOffThreads - 1) / kOffThreads;
    const int i0 = min(n, tid * per), i1 = min(n, i0 + per);
    auto items = [&](int i) -> int32_t {
      if (i == c) return 0;
      const int p = order[i];
      const int64_t m = pair_off[p + 1] - pair_off[p];
      return (int32_t)((m + qb - 1) / qb);
    };
    int32_t sum = 0;
    for (int i = i0; i < i1; ++i) sum += items(i);
    int32_t total;
    int32_t run = block_exclusive_scan<int32_t>(sum, warp32, total);
    for (int i = i0; i < i1; ++i) {
      item_base[i] = run;
      run += items(i);
      cursor[i] = 0;
    }
  }
}

// ------------------------------------------------------------ scan

struct BruteWork {
  int64_t n, nq, rb;
  int nrc, qb;
  __device__ int count() const { return (int)(((nq + qb - 1) / qb) * nrc); }
  __device__ void describe(int item, int64_t& r0, int64_t& r1, int64_t& e0, int& nqi) const {
    int64_t qc = item / nrc, rc = item % nrc;
    e0 = qc * qb * nrc + rc;        // encodes (first query, row chunk)
    nqi = (int)min((int64_t)qb, nq - qc * qb);
    r0 = rc * rb;
    r1 = min(n, r0 + rb);
  }
  // local slot i of an item whose e0 encodes (q0 * nrc + rc): e = e0 + i * nrc
  __device__ int64_t query(int64_t e) const { return e / nrc; }
  __device__ int64_t slot(int64_t e) const { return e; }
};

template <typename W> struct Stride { static constexpr bool v = false; };
template <> struct Stride<BruteWork> { static constexpr bool v = true; };

template <typename RowT, typename Work>
__global__ void __launch_bounds__(kThreads) scan_kernel(
    Work work, int step_nrc, const RowT* __restrict__ rows, int row_stride, const int32_t* __restrict__ row_ids,
    const float* __restrict__ row_scales, const float* __restrict__ Qf, const float* __restrict__ qscale,
    int xs, int k, int qb, int* __restrict__ counter, Cand* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* Qs = reinterpret_cast<float*>(smem);          // [QB][xs]
  float* Xs = Qs + QB * xs;                            // [RB][xs]
  float* Ss = Xs + RB * xs;                            // [QB][SSTRIDE]
  Cand* lists = reinterpret_cast<Cand*>(Ss + QB * SSTRIDE);  // [qb][k]
  int32_t* ids_s = reinterpret_cast<int32_t*>(lists + qb * k);  // [RB]
  float* rsc_s = reinterpret_cast<float*>(ids_s + RB);          // [RB]
  float* qsc_s = rsc_s + RB;                                    // [QB]
  __shared__ int item_s;

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int d4 = row_stride * sizeof(RowT) / 16 * Expand<RowT>::kPer / 4;   // float4 steps per row
  const int cpr = row_stride * (int)sizeof(RowT) / 16;                      // uint4 chunks per row
  const int total = work.count();
  const bool strided = Stride<Work>::v;

  for (;;) {
    if (tid == 0) item_s = atomicAdd(counter, 1);
    __syncthreads();
    const int item = item_s;
    __syncthreads();
    if (item >= total) break;
    int64_t r0, r1, e0;
    int nqi;
    work.describe(item, r0, r1, e0, nqi);
    // queries of this item
    for (int idx = tid; idx < QB * (xs / 4); idx += kThreads) {
      int i = idx / (xs / 4), c4 = idx % (xs / 4);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < nqi && c4 < d4) {
        int64_t e = strided ? e0 + (int64_t)i * step_nrc : e0 + i;
        v = *reinterpret_cast<const float4*>(Qf + work.query(e) * (int64_t)(d4 * 4) + c4 * 4);
      }
      *reinterpret_cast<float4*>(Qs + i * xs + c4 * 4) = v;
    }
    if (tid < QB) {
      float sc = 1.f;
      if (qscale && tid < nqi) {
        int64_t e = strided ? e0 + (int64_t)tid * step_nrc : e0 + tid;
        sc = qscale[work.query(e)];
      }
      qsc_s[tid] = sc;
    }
    for (int idx = tid; idx < qb * k; idx += kThreads) lists[idx] = Cand{-INFINITY, -1};

    for (int64_t t0 = r0; t0 < r1; t0 += RB) {
      const int nr = (int)min((int64_t)RB, r1 - t0);
      __syncthreads();
      const uint4* src = reinterpret_cast<const uint4*>(rows + t0 * row_stride);
      for (int ch = tid; ch < RB * cpr; ch += kThreads) {
        int r = ch / cpr, cc = ch % cpr;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r < nr) v = src[(int64_t)r * cpr + cc];
        Expand<RowT>::to(v, Xs + r * xs + cc * Expand<RowT>::kPer);
      }
      if (tid < RB) {
        ids_s[tid] = tid < nr ? (row_ids ? row_ids[t0 + tid] : (int32_t)(t0 + tid)) : -1;
        rsc_s[tid] = (row_scales && tid < nr) ? row_scales[t0 + tid] : 1.f;
      }
      __syncthreads();
      float acc[4][4] = {};
      for (int k4 = 0; k4 < d4; ++k4) {
        float4 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const float4*>(Qs + (ty * 4 + i) * xs + k4 * 4);
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = *reinterpret_cast<const float4*>(Xs + (tx + 16 * j) * xs + k4 * 4);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float s = acc[i][j];
            s = fmaf(a[i].x, b[j].x, s);
            s = fmaf(a[i].y, b[j].y, s);
            s = fmaf(a[i].z, b[j].z, s);
            s = fmaf(a[i].w, b[j].w, s);
            acc[i][j] = s;
          }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int qi = ty * 4 + i, rj = tx + 16 * j;
          float v = acc[i][j];
          if (row_scales) v = v * qsc_s[qi] * rsc_s[rj];
          Ss[qi * SSTRIDE + rj] = v;
        }
      __syncthreads();
      // per-query top-k: 4 threads per query pre-filter 16 rows each against
      // the current k-th entry, then insert their survivors in turn
      {
        const int qi = tid >> 2, sub = tid & 3;
        unsigned pass = 0;
        if (qi < nqi) {
          Cand worst = lists[qi * k + k - 1];
#pragma unroll
          for (int m = 0; m < 16; ++m) {
            int r = sub + 4 * m;
            if (r < nr && better(Ss[qi * SSTRIDE + r], ids_s[r], worst.s, worst.id)) pass |= 1u << m;
          }
        }
        for (int turn = 0; turn < 4; ++turn) {
          if (sub == turn) {
            while (pass) {
              int m = __ffs(pass) - 1;
              pass &= pass - 1;
              int r = sub + 4 * m;
              float s = Ss[qi * SSTRIDE + r];
              int id = ids_s[r];
              Cand* L = lists + qi * k;
              if (!better(s, id, L[k - 1].s, L[k - 1].id)) continue;
              int pos = k - 1;
              while (pos > 0 && better(s, id, L[pos - 1].s, L[pos - 1].id)) {
                L[pos] = L[pos - 1];
                --pos;
              }
              L[pos] = Cand{s, id};
            }
          }
          __syncwarp();
        }
      }
    }
    __syncthreads();
    for (int idx = tid; idx < nqi * k; idx += kThreads) {
      int i = idx / k, j = idx % k;
      int64_t e = strided ? e0 + (int64_t)i * step_nrc : e0 + i;
      partials[work.slot(e) * k + j] = lists[i * k + j];
    }
  }
}

// ------------------------------------------------------------ merge

// Warp per query: k-way merge of its lists (each sorted best first, length
// `len`, id -1 marks an exhausted tail), dropping a candidate equal in
// (score, id) to the one emitted just before it.
template <bool kIvf>
__global__ void __launch_bounds__(128) merge_kernel(const Cand* __restrict__ partials, int len, int64_t nq,
                                                    int tmax, const int32_t* __restrict__ tpq,
                                                    const int32_t* __restrict__ inv, int nrc, int kout,
                                                    int64_t* __restrict__ ids64, int32_t* __restrict__ ids32,
                                                    float* __restrict__ scores) {
  extern __shared__ uint16_t heads_all[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * 4 + w;
  if (q >= nq) return;
  const int nl = kIvf ? (tpq ? min(max(tpq[q], 0), tmax) : tmax) : nrc;
  uint16_t* head = heads_all + w * (kIvf ? tmax : nrc);
  for (int j = lane; j < nl; j += 32) head[j] = 0;
  __syncwarp();
  auto list_ptr = [&](int j) -> const Cand* {
    int64_t slot = kIvf ? (int64_t)inv[q * tmax + j] : q * nrc + j;
    return partials + slot * len;
  };
  auto lane_best = [&](float& bs, int& bid, int& bj) {
    bs = -INFINITY;
    bid = -1;
    bj = -1;
    for (int j = lane; j < nl; j += 32) {
      int h = head[j];
      if (h >= len) continue;
      Cand c = list_ptr(j)[h];
      if (c.id < 0) continue;
      if (bj < 0 || better(c.s, c.id, bs, bid)) { bs = c.s; bid = c.id; bj = j; }
    }
  };
  float bs;
  int bid, bj;
  lane_best(bs, bid, bj);
  int emitted = 0;
  float last_s = 0.f;
  int last_id = -1;
  while (emitted < kout) {
    float ws = bs;
    int wid = bid, wl = bj >= 0 ? lane : 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float os = __shfl_xor_sync(0xffffffffu, ws, o);
      int oid = __shfl_xor_sync(0xffffffffu, wid, o);
      int ol = __shfl_xor_sync(0xffffffffu, wl, o);
      bool take;
      if (ol == 32) take = false;
      else if (wl == 32) take = true;
      else take = better(os, oid, ws, wid) || (os == ws && oid == wid && ol < wl);
      if (take) { ws = os; wid = oid; wl = ol; }
    }
    if (wl == 32) break;   // every list exhausted
    if (!(emitted > 0 && ws == last_s && wid == last_id)) {
      if (lane == 0) {
        if (ids64) ids64[q * kout + emitted] = wid;
        if (ids32) ids32[q * kout + emitted] = wid;
        if (scores) scores[q * kout + emitted] = ws;
      }
      ++emitted;
      last_s = ws;
      last_id = wid;
    }
    if (lane == wl) {
      head[bj] = head[bj] + 1;
      lane_best(bs, bid, bj);
    }
    __syncwarp();
  }
  for (int i = emitted + lane; i < kout; i += 32) {
    if (ids64) ids64[q * kout + i] = -1;
    if (ids32) ids32[q * kout + i] = -1;
    if (scores) scores[q * kout + i] = -INFINITY;
  }
}

// ------------------------------------------------------------ exact rescoring

// Warp per query: exact fp32 <q, x> of each candidate from the single stored
// copy, then the best k by repeated warp arg-max (candidates are distinct).
template <typename OT, typename QT>
__global__ void __launch_bounds__(128) rescore_kernel(const int32_t* __restrict__ cand, int R, int64_t nq,
                                                      const QT* __restrict__ Q, int d, const OT* __restrict__ orig,
                                                      int ostride, int k, float* __restrict__ work,
                                                      int64_t* __restrict__ ids_out, float* __restrict__ s_out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * 4 + w;
  if (q >= nq) return;
  float* ws = work + q * R;
  const int32_t* cq = cand + q * R;
  for (int i = lane; i < R; i += 32) {
    int id = cq[i];
    float s = -INFINITY;
    if (id >= 0) {
      s = 0.f;
      const OT* x = orig + (int64_t)id * ostride;
      for (int kk = 0; kk < d; ++kk) s = fmaf(load_elem(Q, q * d + kk), load_elem(x, kk), s);
    }
    ws[i] = s;
  }
  __syncwarp();
  for (int out = 0; out < k; ++out) {
    float bs = -INFINITY;
    int bid = -1, bi = -1;
    for (int i = lane; i < R; i += 32) {
      int id = cq[i];
      if (id < 0) continue;
      float s = ws[i];
      if (bi < 0 || better(s, id, bs, bid)) { bs = s; bid = id; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float os = __shfl_xor_sync(0xffffffffu, bs, o);
      int oid = __shfl_xor_sync(0xffffffffu, bid, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      bool take = oi >= 0 && (bi < 0 || better(os, oid, bs, bid));
      if (take) { bs = os; bid = oid; bi = oi; }
    }
    if (lane == 0) {
      ids_out[q * k + out] = bi >= 0 ? bid : -1;
      s_out[q * k + out] = bi >= 0 ? bs : -INFINITY;
    }
    if (bi >= 0 && lane == (bi & 31)) ws[bi] = -INFINITY, const_cast<int32_t*>(cq)[bi] = -1;
    __syncwarp();
  }
}

// ------------------------------------------------------------ host glue

int scan_smem_bytes(int xs, int k, int qb) {
  return (QB * xs + RB * xs + QB * SSTRIDE) * 4 + qb * k * (int)sizeof(Cand) + RB * 8 + QB * 4;
}

// Query slots per work item: 64, fewer when the per-query lists would not fit.
int scan_qb(int xs, int k) {
  const int budget = 200 * 1024;
  int qb = QB;
  while (qb > 1 && scan_smem_bytes(xs, k, qb) > budget) qb = qb > 4 ? qb - 4 : qb - 1;
  return qb;
}

template <typename RowT>
int scan_xs(int row_stride) { return smem_stride(row_stride * (int)sizeof(RowT) / 16 * Expand<RowT>::kPer); }

template <typename RowT, typename Work>
void launch_scan(const Work& work, int step_nrc, int max_items, const RowT* rows, int row_stride,
                 const int32_t* row_ids, const float* row_scales, const float* Qf, const float* qscale, int k,
                 int qb, Cand* partials, cudaStream_t s, Scratch& scr) {
  const int xs = scan_xs<RowT>(row_stride);
  const int smem = scan_smem_bytes(xs, k, qb);
  auto kern = scan_kernel<RowT, Work>;
  SOAR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  SOAR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  if (per_sm < 1) fail(SOAR_EUNSUPPORTED, "scan: shared memory for k too large");
  int grid = std::max(1, std::min(max_items, per_sm * num_sms()));
  int* counter = scr.get<int>(1);
  SOAR_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), s));
  stage_mark(s, "scan", true);
  kern<<<grid, kThreads, smem, s>>>(work, step_nrc, rows, row_stride, row_ids, row_scales, Qf, qscale, xs, k,
                                    qb, counter, partials);
  SOAR_LAUNCHED();
  stage_mark(s, "scan", false);
}

template <typename QT>
void prep(const QT* Q, int64_t nq, int d, int stride, bool fp8, float* Qf, float* qscale, float* qnorm,
          cudaStream_t s) {
  prep_queries<QT><<<ceil_div(nq * 32, 256), 256, 0, s>>>(Q, nq, d, stride, fp8, Qf, qscale, qnorm);
  SOAR_LAUNCHED();
}

void prep_any(const void* Q, soar_dtype dt, int64_t nq, int d, int stride, bool fp8, float* Qf, float* qscale,
              cudaStream_t s, float* qnorm = nullptr) {
  if (dt == SOAR_F32) prep<float>(static_cast<const float*>(Q), nq, d, stride, fp8, Qf, qscale, qnorm, s);
  else prep<__nv_bfloat16>(static_cast<const __nv_bfloat16*>(Q), nq, d, stride, fp8, Qf, qscale, qnorm, s);
}

int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// S = Q . C^T for prepared queries (FP8 indices: scaled code products).
void score_centroids(const IndexData& ix, const float* Qf, const float* qscale, int64_t nq, int qstride, float* S,
                     cudaStream_t s) {
  const bool fp8 = ix.mode == SOAR_SCORE_FP8;
  const float* B = fp8 ? ix.cent_code_vals : ix.centroids;
  const int ldb = fp8 ? ix.code_stride : ix.d;
  const bool aligned = qstride % 4 == 0 && ldb % 4 == 0 && (reinterpret_cast<uintptr_t>(Qf) & 15u) == 0 &&
                       (reinterpret_cast<uintptr_t>(B) & 15u) == 0;
  if (aligned) {
    dim3 grid(ceil_div(ix.c, 128), ceil_div(nq, 128));
    gemm_nt_128<<<grid, 256, 0, s>>>(Qf, nq, qstride, B, ix.c, ldb, ix.d, fp8 ? qscale : nullptr,
                                     fp8 ? ix.cent_scales : nullptr, S);
  } else {
    dim3 grid(ceil_div(ix.c, 64), ceil_div(nq, 64));
    gemm_nt<<<grid, 256, 0, s>>>(Qf, nq, qstride, B, ix.c, ldb, ix.d, fp8 ? qscale : nullptr,
                                 fp8 ? ix.cent_scales : nullptr, S);
  }
  SOAR_LAUNCHED();
}

// Queries already prepared (Qf, row stride qstride); writes top [nq][t].
void select_prepared(const IndexData& ix, const float* Qf, const float* qscale, int64_t nq, int qstride, int t,
                     int32_t* top, float* top_s, cudaStream_t s, Scratch& scr) {
  if (!qscale && select_tc_usable(ix, Qf, qstride, t)) {
    select_tc(ix, Qf, nq, qstride, t, top, top_s, s);   // scores and top-t fused on the tensor cores
    return;
  }
  float* S = scr.get<float>((size_t)nq * ix.c);
  score_centroids(ix, Qf, qscale, nq, qstride, S, s);
  if (t <= 32) {
    topt_warp_kernel<<<ceil_div(nq * 32, 256), 256, 0, s>>>(S, nq, ix.c, t, top, top_s);
    SOAR_LAUNCHED();
    return;
  }
  const int t2 = pow2_at_least(t);
  const int smem = t2 * 8 + (ix.c <= kToptSmemRow ? ix.c * 4 : 0);
  SOAR_CUDA(cudaFuncSetAttribute(topt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  topt_kernel<<<(unsigned)nq, 256, smem, s>>>(S, ix.c, t, t2, top, top_s);
  SOAR_LAUNCHED();
}

struct Grouped {
  const int32_t* order;    // [c] partitions in the order their items are handed out
  int64_t* pair_off;       // [c + 1]
  const int32_t* vals;     // pairs sorted by partition (value q * t + j)
  int32_t* item_base;      // [c + 1]
  int max_items;
};

// (query, probe) pairs grouped by partition (counting sort), the inverse
// map inv[q * t + j] = grouped position, and the work items (partition,
// <= qb pairs) counted over partitions in size order.
Grouped group_pairs(const IndexData& ix, int64_t nq, int t, const int32_t* tpq, int qb, const int32_t* top,
                    int32_t* inv, cudaStream_t s, Scratch& scr, bool first_probes_first = false) {
  const int64_t P = nq * t;
  const int c = ix.c;
  stage_mark(s, "group", true);
  // the pair counts [c + 2], then (first-probe order only) the first-probe
  // counts [c] in the same allocation, cleared by one memset
  const bool by_first = first_probes_first && c <= kRankMaxC;
  const size_t words = (size_t)c + 2 + (by_first ? ((size_t)c + 1) / 2 : 0);
  unsigned long long* cnt = scr.get<unsigned long long>(words);
  int32_t* cursor = scr.get<int32_t>((size_t)c + 1);
  SOAR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * words, s));
  unsigned* first = by_first ? reinterpret_cast<unsigned*>(cnt + c + 2) : nullptr;
  pair_counts<<<ceil_div(P, 256), 256, 0, s>>>(top, nq, t, tpq, c, cnt, first);
  SOAR_LAUNCHED();
  Grouped g;
  g.order = ix.part_order;
  if (first) {
    int32_t* order = scr.get<int32_t>(c);
    first_probe_order<<<ceil_div(c, 32), 256, 0, s>>>(ix.part_order, first, c, order);
    SOAR_LAUNCHED();
    g.order = order;
  }
  g.pair_off = scr.get<int64_t>((size_t)c + 2);
  g.item_base = scr.get<int32_t>((size_t)c + 1);
  group_offsets<<<1, kOffThreads, 0, s>>>(cnt, c, g.order, qb, g.pair_off, g.item_base, cursor);
  SOAR_LAUNCHED();
  int32_t* vals = scr.get<int32_t>(P);
  pair_scatter<<<ceil_div(P, 256), 256, 0, s>>>(top, nq, t, tpq, c, g.pair_off, cursor, vals, inv);
  SOAR_LAUNCHED();
  stage_mark(s, "group", false);
  g.vals = vals;
  g.max_items = (int)std::min<int64_t>(P / qb + c + 1, 1 << 30);
  return g;
}

template <typename RowT>
void ivf_scan_typed(const IndexData& ix, const float* Qf, const float* qscale, int64_t nq, int t,
                    const int32_t* tpq, int len, Cand* partials, int32_t* inv, const int32_t* top,
                    cudaStream_t s, Scratch& scr) {
  const int qb = scan_qb(scan_xs<RowT>(ix.row_stride), len);
  Grouped g = group_pairs(ix, nq, t, tpq, qb, top, inv, s, scr);
  IvfWork work{ix.offsets, g.pair_off, g.vals, g.order, g.item_base, ix.c, t, qb};
  launch_scan<RowT, IvfWork>(work, 1, g.max_items, static_cast<const RowT*>(ix.vectors), ix.row_stride, ix.ids,
                             ix.row_scales, Qf, qscale, len, qb, partials, s, scr);
}

}  // namespace

void centroid_scores(const IndexData& ix, const void* Q, soar_dtype dt, int64_t nq, float* S, cudaStream_t s,
                     Scratch& scr) {
  const bool fp8 = ix.mode == SOAR_SCORE_FP8;
  const int qstride = fp8 ? ix.code_stride : (ix.d + 3) / 4 * 4;
  float* Qf = scr.get<float>((size_t)nq * qstride);
  float* qscale = fp8 ? scr.get<float>(nq) : nullptr;
  prep_any(Q, dt, nq, ix.d, qstride, fp8, Qf, qscale, s);
  score_centroids(ix, Qf, qscale, nq, qstride, S, s);
}

void select_partitions(const IndexData& ix, const void* Q, soar_dtype dt, int64_t nq, int32_t t, int32_t* top,
                       float* top_scores, cudaStream_t s, Scratch& scr) {
  const bool fp8 = ix.mode == SOAR_SCORE_FP8;
  const int qstride = fp8 ? ix.code_stride : (ix.d + 3) / 4 * 4;
  float* Qf = scr.get<float>((size_t)nq * qstride);
  float* qscale = fp8 ? scr.get<float>(nq) : nullptr;
  prep_any(Q, dt, nq, ix.d, qstride, fp8, Qf, qscale, s);
  select_prepared(ix, Qf, qscale, nq, qstride, t, top, top_scores, s, scr);
}

size_t select_scratch_bytes(const IndexData& ix, int64_t nq) {
  const bool fp8 = ix.mode == SOAR_SCORE_FP8;
  const int qstride = fp8 ? ix.code_stride : (ix.d + 3) / 4 * 4;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  return up(sizeof(float) * (size_t)nq * qstride) + up(fp8 ? sizeof(float) * (size_t)nq : 0) +
         up(sizeof(float) * (size_t)nq * ix.c);
}

void select_partitions_in(const IndexData& ix, const void* Q, soar_dtype dt, int64_t nq, int32_t t, int32_t* top,
                          float* top_scores, void* scratch, cudaStream_t s) {
  const bool fp8 = ix.mode == SOAR_SCORE_FP8;
  const int qstride = fp8 ? ix.code_stride : (ix.d + 3) / 4 * 4;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  char* base = static_cast<char*>(scratch);
  float* Qf = reinterpret_cast<float*>(base);
  base += up(sizeof(float) * (size_t)nq * qstride);
  float* qscale = fp8 ? reinterpret_cast<float*>(base) : nullptr;
  base += up(fp8 ? sizeof(float) * (size_t)nq : 0);
  float* S = reinterpret_cast<float*>(base);
  // every scratch element read below is first written here: nothing to clear
  prep_any(Q, dt, nq, ix.d, qstride, fp8, Qf, qscale, s);
  if (!fp8 && select_tc_usable(ix, Qf, qstride, t)) {
    select_tc(ix, Qf, nq, qstride, t, top, top_scores, s);   // needs no scratch beyond Qf
    return;
  }
  score_centroids(ix, Qf, qscale, nq, qstride, S, s);
  const int t2 = pow2_at_least(t);
  const int smem = t2 * 8 + (ix.c <= kToptSmemRow ? ix.c * 4 : 0);
  SOAR_CUDA(cudaFuncSetAttribute(topt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  topt_kernel<<<(unsigned)nq, 256, smem, s>>>(S, ix.c, t, t2, top, top_scores);
  SOAR_LAUNCHED();
}

// Fine probes from an IVF search over the fine centroids: its ids (int64,
// best first, -1 padding after the last one found) become int32 partition
// ids, and the number found is the query's probe count.  Entry e = q * t + j
// writes top[e]; the last entry found (or j = 0 when none is) writes the count.
__global__ void fine_probes(const int64_t* __restrict__ ids, int64_t total, int t, int32_t* __restrict__ top,
                            int32_t* __restrict__ count) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int64_t q = e / t;
  const int j = (int)(e - q * t);
  const int64_t v = ids[e];
  top[e] = v >= 0 ? (int32_t)v : -1;
  if (v >= 0 && (j == t - 1 || ids[e + 1] < 0)) count[q] = j + 1;
  if (j == 0 && v < 0) count[q] = 0;
}

void multilevel_select(const IndexData& coarse, const void* Q, soar_dtype dt, int64_t nq, int32_t t, int32_t t1,
                       int32_t* top, float* top_scores, int32_t* count, cudaStream_t s, Scratch& scr) {
  int64_t* ids = scr.get<int64_t>((size_t)nq * t);
  float* sc = top_scores ? top_scores : scr.get<float>((size_t)nq * t);
  search(coarse, Q, dt, nq, t, t1, nullptr, 0, ids, sc, s, scr);
  fine_probes<<<ceil_div(nq * t, 256), 256, 0, s>>>(ids, nq * t, t, top, count);
  SOAR_LAUNCHED();
}

// The search's selection with the learned probe count: the top t with their
// scores, the features [q || scores], the network's per-query counts.
static const int32_t* learned_select(const IndexData& ix, const void* Q, soar_dtype dt, const float* Qf,
                                     const float* qscale, int64_t nq, int qstride, int t, const LearnedProbe& lp,
                                     int32_t* top, cudaStream_t s, Scratch& scr) {
  float* top_s = scr.get<float>((size_t)nq * t);
  select_prepared(ix, Qf, qscale, nq, qstride, t, top, top_s, s, scr);
  float* Z = scr.get<float>((size_t)nq * (ix.d + t));
  features_from_scores(Q, dt, nq, ix.d, top_s, t, Z, s);
  int32_t* tq = lp.t_out ? lp.t_out : scr.get<int32_t>(nq);
  mlp_predict(lp.params, lp.d_in, lp.hidden, Z, (int)nq, lp.bf16, lp.alpha, lp.t_cap, nullptr, tq, s, scr);
  return tq;
}

void search(const IndexData& ix, const void* Q, soar_dtype dt, int64_t nq, int32_t k, int32_t t,
            const int32_t* tpq, int32_t rescore, int64_t* ids_out, float* scores_out, cudaStream_t s,
            Scratch& scr, const IndexData* coarse, int32_t t1, const LearnedProbe* learned) {
  const bool fp8 = ix.mode == SOAR_SCORE_FP8;
  if (!fp8 && ix.tc_rows && k <= scan_tc_max_k(ix)) {
    // fp32 index: tensor-core screening with exact fp32 rescoring
    const int qstride = ix.tc_kp;
    float* Qf = scr.get<float>((size_t)nq * qstride);
    float* qn = scr.get<float>(nq);
    stage_mark(s, "select", true);
    prep_any(Q, dt, nq, ix.d, qstride, false, Qf, nullptr, s, qn);   // rows and their norms
    int32_t* top = scr.get<int32_t>((size_t)nq * t);
    if (coarse) {
      int32_t* found = scr.get<int32_t>(nq);
      multilevel_select(*coarse, Q, dt, nq, t, t1, top, nullptr, found, s, scr);
      tpq = found;
    } else if (learned) {
      tpq = learned_select(ix, Q, dt, Qf, nullptr, nq, qstride, t, *learned, top, s, scr);
    } else {
      select_prepared(ix, Qf, nullptr, nq, qstride, t, top, nullptr, s, scr);
    }
    stage_mark(s, "select", false);
    if (scan_by_query_usable(ix, nq, t, k)) {   // few queries per probed partition: query-major exact scan
      Cand* lists = scr.get<Cand>((size_t)nq * t * k);
      stage_mark(s, "scan", true);
      scan_by_query(ix, Qf, qstride, top, tpq, nq, t, k, lists, s);
      stage_mark(s, "scan", false);
      // k-way merge of each query's t lists; a spilled copy repeats (score, id) and is dropped
      const int smem = 4 * t * (int)sizeof(uint16_t);
      SOAR_CUDA(cudaFuncSetAttribute(merge_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      stage_mark(s, "merge", true);
      merge_kernel<false><<<ceil_div(nq, 4), 128, smem, s>>>(lists, k, nq, 0, nullptr, nullptr, t, k, ids_out,
                                                             nullptr, scores_out);
      SOAR_LAUNCHED();
      stage_mark(s, "merge", false);
      return;
    }
    const int64_t P = nq * t;
    int32_t* inv = scr.get<int32_t>(P);
    const int len = scan_tc_list_len(k);
    Cand* lists = scr.get<Cand>((size_t)P * len);
    Grouped g = group_pairs(ix, nq, t, tpq, 128, top, inv, s, scr, true);
    IvfWork work{ix.offsets, g.pair_off, g.vals, g.order, g.item_base, ix.c, t, 128};
    if (scan_tc_search(ix, work, g.max_items, Qf, qn, top, inv, tpq, nq, t, k, lists, device_error_word(), ids_out,
                       scores_out, s, scr))
      return;                                   // rescored and merged by the scan's finishing kernel
    const int smem = 4 * t * (int)sizeof(uint16_t);
    SOAR_CUDA(cudaFuncSetAttribute(merge_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    stage_mark(s, "merge", true);
    merge_kernel<true><<<ceil_div(nq, 4), 128, smem, s>>>(lists, len, nq, t, tpq, inv, 0, k, ids_out, nullptr,
                                                          scores_out);
    SOAR_LAUNCHED();
    stage_mark(s, "merge", false);
    return;
  }
  // query rows padded exactly like the index rows (float elements); a PQ4
  // index scores fp32 query rows against fp32 centroids and its LUTs
  const bool pq = ix.mode == SOAR_SCORE_PQ4;
  int qstride;
  if (fp8) qstride = ix.code_stride;
  else if (pq) qstride = (ix.d + 3) / 4 * 4;
  else qstride = ix.row_stride;            // fp32 or bf16 rows: row_stride elements
  float* Qf = scr.get<float>((size_t)nq * qstride);
  float* qscale = fp8 ? scr.get<float>(nq) : nullptr;
  stage_mark(s, "select", true);
  prep_any(Q, dt, nq, ix.d, qstride, fp8, Qf, qscale, s);
  int32_t* top = scr.get<int32_t>((size_t)nq * t);
  if (coarse) {
    int32_t* found = scr.get<int32_t>(nq);
    multilevel_select(*coarse, Q, dt, nq, t, t1, top, nullptr, found, s, scr);
    tpq = found;
  } else if (learned) {
    tpq = learned_select(ix, Q, dt, Qf, qscale, nq, qstride, t, *learned, top, s, scr);
  } else {
    select_prepared(ix, Qf, qscale, nq, qstride, t, top, nullptr, s, scr);
  }
  stage_mark(s, "select", false);
  if (!fp8 && !pq) {
    const int64_t P = nq * t;
    int32_t* inv = scr.get<int32_t>(P);
    Cand* partials = scr.get<Cand>((size_t)P * k);
    if (ix.dtype == SOAR_F32)
      ivf_scan_typed<float>(ix, Qf, qscale, nq, t, tpq, k, partials, inv, top, s, scr);
    else
      ivf_scan_typed<__nv_bfloat16>(ix, Qf, qscale, nq, t, tpq, k, partials, inv, top, s, scr);
    const int smem = 4 * t * (int)sizeof(uint16_t);
    SOAR_CUDA(cudaFuncSetAttribute(merge_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    stage_mark(s, "merge", true);
    merge_kernel<true><<<ceil_div(nq, 4), 128, smem, s>>>(partials, k, nq, t, tpq, inv, 0, k, ids_out, nullptr,
                                                          scores_out);
    SOAR_LAUNCHED();
    stage_mark(s, "merge", false);
    return;
  }
  // FP8 / PQ4: the best `rescore` approximate scores of each query's probed
  // union (each point once), rescored exactly in fp32 from the stored rows.
  int32_t* cand = scr.get<int32_t>((size_t)nq * rescore);
  stage_mark(s, "scan", true);
  if (fp8)
    fp8_shortlist(ix, Qf, qscale, top, tpq, nq, t, rescore, cand, s, scr);
  else
    pq_shortlist(ix, Qf, qstride, top, tpq, nq, t, rescore, cand, s, scr);
  stage_mark(s, "scan", false);
  float* work = scr.get<float>((size_t)nq * rescore);
  const int ostride = ix.dtype == SOAR_F32 ? (ix.d + 3) / 4 * 4 : (ix.d + 7) / 8 * 8;
  if (ix.dtype == SOAR_F32) {
    if (dt == SOAR_F32)
      rescore_kernel<float, float><<<ceil_div(nq, 4), 128, 0, s>>>(cand, rescore, nq, static_cast<const float*>(Q),
          ix.d, static_cast<const float*>(ix.originals), ostride, k, work, ids_out, scores_out);
    else
      rescore_kernel<float, __nv_bfloat16><<<ceil_div(nq, 4), 128, 0, s>>>(cand, rescore, nq,
          static_cast<const __nv_bfloat16*>(Q), ix.d, static_cast<const float*>(ix.originals), ostride, k, work,
          ids_out, scores_out);
  } else {
    if (dt == SOAR_F32)
      rescore_kernel<__nv_bfloat16, float><<<ceil_div(nq, 4), 128, 0, s>>>(cand, rescore, nq,
          static_cast<const float*>(Q), ix.d, static_cast<const __nv_bfloat16*>(ix.originals), ostride, k, work,
          ids_out, scores_out);
    else
      rescore_kernel<__nv_bfloat16, __nv_bfloat16><<<ceil_div(nq, 4), 128, 0, s>>>(cand, rescore, nq,
          static_cast<const __nv_bfloat16*>(Q), ix.d, static_cast<const __nv_bfloat16*>(ix.originals), ostride, k,
          work, ids_out, scores_out);
  }
  SOAR_LAUNCHED();
}

namespace {
// (id + id_offsets[list], score) of every list entry as merge candidates.
__global__ void pack_lists(const int64_t* __restrict__ ids, const float* __restrict__ scores, int64_t count, int m,
                           int len, const int64_t* __restrict__ id_offsets, Cand* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int64_t id = ids[i];
  const int list = (int)((i / len) % m);
  out[i] = id < 0 ? Cand{-INFINITY, -1} : Cand{scores[i], (int32_t)(id + (id_offsets ? id_offsets[list] : 0))};
}
}  // namespace

void merge_topk(const int64_t* ids, const float* scores, int64_t nq, int m, int len, const int64_t* id_offsets,
                int k, int64_t* ids_out, float* scores_out, cudaStream_t s, Scratch& scr) {
  const int64_t count = nq * m * (int64_t)len;
  Cand* c = scr.get<Cand>((size_t)count);
  pack_lists<<<ceil_div(count, 256), 256, 0, s>>>(ids, scores, count, m, len, id_offsets, c);
  SOAR_LAUNCHED();
  const int smem = 4 * m * (int)sizeof(uint16_t);
  SOAR_CUDA(cudaFuncSetAttribute(merge_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  merge_kernel<false><<<ceil_div(nq, 4), 128, smem, s>>>(c, len, nq, 0, nullptr, nullptr, m, k, ids_out, nullptr,
                                                         scores_out);
  SOAR_LAUNCHED();
}

void exact_mips(const void* X, soar_dtype xdt, int64_t n, int32_t d, const void* Q, soar_dtype qdt, int64_t nq,
                int32_t k, int64_t* ids_out, float* scores_out, cudaStream_t s, Scratch& scr) {
  const size_t esz = xdt == SOAR_F32 ? 4 : 2;
  const int stride = (int)(((d * esz + 15) / 16) * 16 / esz);
  const void* rows = X;
  if (stride != d || (reinterpret_cast<uintptr_t>(X) & 15u)) {
    // padded copy so every row starts on a 16-byte boundary
    void* pad = scr.get<unsigned char>(esz * (size_t)n * stride);
    SOAR_CUDA(cudaMemcpy2DAsync(pad, esz * stride, X, esz * d, esz * d, n, cudaMemcpyDeviceToDevice, s));
    if (stride != d)
      SOAR_CUDA(cudaMemset2DAsync(static_cast<unsigned char*>(pad) + esz * d, esz * stride, 0, esz * (stride - d), n, s));
    rows = pad;
  }
  // Tensor-core path: the rows become a flat index of 65 536-row chunks that
  // every query probes, so the partition scan (tensor-core screening with
  // exact fp32 finishing) returns the exact top k of all rows.
  {
    constexpr int64_t kChunkRows = 65536;
    IndexData fx;
    fx.n = n;
    fx.rows = n;
    fx.d = d;
    fx.dtype = xdt;
    fx.mode = SOAR_SCORE_F32;
    fx.row_stride = stride;
    fx.vectors = const_cast<void*>(rows);
    fx.c = (int)((n + kChunkRows - 1) / kChunkRows);
    const int kstep = xdt == SOAR_F32 ? 8 : 16;
    fx.tc_kp = (d + kstep - 1) / kstep * kstep;
    if (k <= scan_tc_max_k(fx)) {
      build_flat_tc(fx, kChunkRows, s, scr);
      const int c = fx.c, len = scan_tc_list_len(k);
      const size_t qesz = qdt == SOAR_F32 ? 4 : 2;
      // queries in batches whose candidate lists stay within about 1 GB
      const int64_t nb = std::max<int64_t>(128, (int64_t(1) << 30) / ((int64_t)c * len * (int64_t)sizeof(Cand)));
      for (int64_t q0 = 0; q0 < nq; q0 += nb) {
        const int64_t m = std::min(nb, nq - q0);
        Scratch bs(s);
        float* Qf = bs.get<float>((size_t)m * fx.tc_kp);
        float* qn = bs.get<float>(m);
        prep_any(static_cast<const char*>(Q) + q0 * d * qesz, qdt, m, d, fx.tc_kp, false, Qf, nullptr, s, qn);
        int32_t* top = bs.get<int32_t>((size_t)m * c);
        all_partitions<<<ceil_div(m * c, 256), 256, 0, s>>>(top, m, c);
        SOAR_LAUNCHED();
        int32_t* inv = bs.get<int32_t>((size_t)m * c);
        Cand* lists = bs.get<Cand>((size_t)m * c * len);
        Grouped g = group_pairs(fx, m, c, nullptr, 128, top, inv, s, bs);
        IvfWork work{fx.offsets, g.pair_off, g.vals, g.order, g.item_base, c, c, 128};
        if (!scan_tc_search(fx, work, g.max_items, Qf, qn, top, inv, nullptr, m, c, k, lists, device_error_word(),
                            ids_out + q0 * k, scores_out + q0 * k, s, bs)) {
          const int smem = 4 * c * (int)sizeof(uint16_t);
          SOAR_CUDA(cudaFuncSetAttribute(merge_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
          merge_kernel<true><<<ceil_div(m, 4), 128, smem, s>>>(lists, len, m, c, nullptr, inv, 0, k,
                                                               ids_out + q0 * k, nullptr, scores_out + q0 * k);
          SOAR_LAUNCHED();
        }
      }
      return;
    }
  }
  // float query rows as wide as the expanded data rows
  const int qstride = stride;
  float* Qf = scr.get<float>((size_t)nq * qstride);
  prep_any(Q, qdt, nq, d, qstride, false, Qf, nullptr, s);
  const int64_t rb = std::max<int64_t>(4096, std::min<int64_t>(65536, (n + 63) / 64));
  const int nrc = (int)((n + rb - 1) / rb);
  Cand* partials = scr.get<Cand>((size_t)nq * nrc * k);
  const int qb = xdt == SOAR_F32 ? scan_qb(scan_xs<float>(stride), k) : scan_qb(scan_xs<__nv_bfloat16>(stride), k);
  BruteWork work{n, nq, rb, nrc, qb};
  const int max_items = (int)(((nq + qb - 1) / qb) * nrc);
  if (xdt == SOAR_F32)
    launch_scan<float, BruteWork>(work, nrc, max_items, static_cast<const float*>(rows), stride, nullptr, nullptr,
                                  Qf, nullptr, k, qb, partials, s, scr);
  else
    launch_scan<__nv_bfloat16, BruteWork>(work, nrc, max_items, static_cast<const __nv_bfloat16*>(rows), stride,
                                          nullptr, nullptr, Qf, nullptr, k, qb, partials, s, scr);
  const int smem = 4 * nrc * (int)sizeof(uint16_t);
  SOAR_CUDA(cudaFuncSetAttribute(merge_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  merge_kernel<false><<<ceil_div(nq, 4), 128, smem, s>>>(partials, k, nq, 0, nullptr, nullptr, nrc, k, ids_out,
                                                         nullptr, scores_out);
  SOAR_LAUNCHED();
}

}  // namespace soar
