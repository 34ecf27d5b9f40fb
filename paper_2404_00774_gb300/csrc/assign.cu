// Primary assignment, SOAR spilled assignment and Lloyd k-means.
//
// Every assignment decision is taken in two stages:
//   screen  -- a tiled X . C^T product scores every (point, centroid) pair
//              with the expanded loss ||c'||^2 - 2<x,c'> + lambda*sum_i(<x,r_i> - <c',r_i>)^2
//              (||x||^2 is constant per point and dropped) and keeps the two
//              best candidates per point; the n x c score matrix never
//              leaves the chip;
//   refine  -- the two candidates are rescored in the direct form
//              ||x - c'||^2 + lambda * sum_i <x - c', r_hat_i>^2 (Theorem 3.1),
//              whose fp32 rounding error is relative to the loss itself, and
//              the smaller wins (lower index on ties).
// If the screen's error were to push the true best out of the top two, the
// two survivors would lie within that error of it, i.e. the decision is a
// near-tie either way.
#include "internal.cuh"

namespace soar {

namespace {

constexpr int kMaxDirs = 4;     // spills supported by the screening kernel
constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
constexpr int kThreads = 256;

__global__ void centroid_norms(const float* C, int c, int d, float* cnorm) {
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= c) return;
  float s = 0.f;
  for (int k = lane; k < d; k += 32) {
    float v = C[(int64_t)w * d + k];
    s = fmaf(v, v, s);
  }
  s = warp_sum(s);
  if (lane == 0) cnorm[w] = s;
}

struct Top2 {
  float b1, b2;
  int i1, i2;
  __device__ void init() { b1 = b2 = INFINITY; i1 = i2 = -1; }
  __device__ static bool better(float a, int ia, float b, int ib) {
    return a < b || (a == b && (unsigned)ia < (unsigned)ib);
  }
  __device__ void push(float v, int i) {
    if (better(v, i, b1, i1)) { b2 = b1; i2 = i1; b1 = v; i1 = i; }
    else if (better(v, i, b2, i2)) { b2 = v; i2 = i; }
  }
};

// Screening kernel.  NDIR = number of residual directions (0 for the
// primary assignment, j for the j-th spill).  Block: 64 points x all
// centroids in tiles of 64; thread (ty, tx) owns 4 points x 4 centroids.
template <int NDIR, typename XT>
__global__ void __launch_bounds__(kThreads) screen_kernel(
    const XT* __restrict__ X, int64_t n, int d, const float* __restrict__ C,
    const float* __restrict__ cnorm, int c, const int32_t* __restrict__ assign, int astride,
    const float* __restrict__ inv_rn, const float* __restrict__ xr, float lambda,
    int32_t* __restrict__ cand) {
  __shared__ __align__(16) float Xs[BK][BM];
  __shared__ __align__(16) float Rs[NDIR > 0 ? NDIR : 1][BK][BM];
  __shared__ __align__(16) float Cs[BK][BN];
  __shared__ int32_t prior_s[BM][kMaxDirs];
  __shared__ float inv_s[BM][kMaxDirs];

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t p0 = (int64_t)blockIdx.x * BM;

  if (NDIR > 0) {
    constexpr int kDiv = NDIR > 0 ? NDIR : 1;
    for (int i = tid; i < BM * NDIR; i += kThreads) {
      int m = i / kDiv, j = i % kDiv;
      int64_t p = p0 + m;
      prior_s[m][j] = p < n ? assign[p * astride + j] : 0;
      inv_s[m][j] = p < n ? inv_rn[p * kMaxDirs + j] : 0.f;
    }
  }
  // per-thread point data for the epilogue
  int32_t prior[TM][kMaxDirs > 0 ? kMaxDirs : 1];
  float xrv[TM][kMaxDirs];
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t p = p0 + ty * TM + i;
#pragma unroll
    for (int j = 0; j < kMaxDirs; ++j) {
      prior[i][j] = (j < NDIR && p < n) ? assign[p * astride + j] : -1;
      xrv[i][j] = (j < NDIR && p < n) ? xr[p * kMaxDirs + j] : 0.f;
    }
  }
  Top2 top[TM];
#pragma unroll
  for (int i = 0; i < TM; ++i) top[i].init();
  __syncthreads();

  for (int c0 = 0; c0 < c; c0 += BN) {
    float ax[TM][TN];
    float ar[NDIR > 0 ? NDIR : 1][TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        ax[i][j] = 0.f;
#pragma unroll
        for (int r = 0; r < (NDIR > 0 ? NDIR : 1); ++r) ar[r][i][j] = 0.f;
      }

    for (int k0 = 0; k0 < d; k0 += BK) {
      __syncthreads();
#pragma unroll
      for (int e = 0; e < (BM * BK) / kThreads; ++e) {
        int idx = tid + e * kThreads;
        int m = idx / BK, kk = idx % BK;
        int64_t p = p0 + m;
        int k = k0 + kk;
        float xv = (p < n && k < d) ? load_elem(X, p * d + k) : 0.f;
        Xs[kk][m] = xv;
#pragma unroll
        for (int r = 0; r < NDIR; ++r) {
          float cv = (p < n && k < d) ? C[(int64_t)prior_s[m][r] * d + k] : 0.f;
          Rs[r][kk][m] = (xv - cv) * inv_s[m][r];
        }
        int cc = c0 + m;
        Cs[kk][m] = (cc < c && k < d) ? C[(int64_t)cc * d + k] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        float4 a = *reinterpret_cast<const float4*>(&Xs[kk][ty * TM]);
        float4 b = *reinterpret_cast<const float4*>(&Cs[kk][tx * TN]);
        float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) ax[i][j] = fmaf(av[i], bv[j], ax[i][j]);
#pragma unroll
        for (int r = 0; r < NDIR; ++r) {
          float4 q = *reinterpret_cast<const float4*>(&Rs[r][kk][ty * TM]);
          float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) ar[r][i][j] = fmaf(qv[i], bv[j], ar[r][i][j]);
        }
      }
    }
    // epilogue: expanded loss and running top-2 per point
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int cc = c0 + tx * TN + j;
      if (cc >= c) continue;
      float cn = cnorm[cc];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        float loss = cn - 2.f * ax[i][j];
        bool taken = false;
#pragma unroll
        for (int r = 0; r < NDIR; ++r) {
          float t = xrv[i][r] - ar[r][i][j];
          loss = fmaf(lambda * t, t, loss);
          taken |= (prior[i][r] == cc);
        }
        if (!taken) top[i].push(loss, cc);
      }
    }
  }
  // merge the 16 partial lists that share these points (lanes differing in tx)
#pragma unroll
  for (int i = 0; i < TM; ++i) {
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
      float ob1 = __shfl_xor_sync(0xffffffffu, top[i].b1, o);
      float ob2 = __shfl_xor_sync(0xffffffffu, top[i].b2, o);
      int oi1 = __shfl_xor_sync(0xffffffffu, top[i].i1, o);
      int oi2 = __shfl_xor_sync(0xffffffffu, top[i].i2, o);
      if (oi1 >= 0) top[i].push(ob1, oi1);
      if (oi2 >= 0) top[i].push(ob2, oi2);
    }
    int64_t p = p0 + ty * TM + i;
    if (tx == 0 && p < n) {
      cand[p * 2 + 0] = top[i].i1;
      cand[p * 2 + 1] = top[i].i2;
    }
  }
}

// For the newest assigned column `dir`: 1/||x - C[a]|| (0 when zero) and <x, r_hat>.
template <typename XT>
__global__ void residual_kernel(const XT* __restrict__ X, int64_t n, int d, const float* __restrict__ C,
                                const int32_t* __restrict__ assign, int astride, int dir,
                                float* __restrict__ inv_rn, float* __restrict__ xr) {
  int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (p >= n) return;
  const float* cr = C + (int64_t)assign[p * astride + dir] * d;
  float ss = 0.f, xd = 0.f;
  for (int k = lane; k < d; k += 32) {
    float xv = load_elem(X, p * d + k);
    float r = xv - cr[k];
    ss = fmaf(r, r, ss);
    xd = fmaf(xv, r, xd);
  }
  ss = warp_sum(ss);
  xd = warp_sum(xd);
  if (lane == 0) {
    float inv = ss > 0.f ? 1.f / sqrtf(ss) : 0.f;
    inv_rn[p * kMaxDirs + dir] = inv;
    xr[p * kMaxDirs + dir] = xd * inv;
  }
}

// Exact direct-form decision between the two screened candidates; writes
// assign[p][col].  col = 0 is the primary assignment (no penalty).
template <typename XT>
__global__ void refine_kernel(const XT* __restrict__ X, int64_t n, int d, const float* __restrict__ C,
                              int32_t* __restrict__ assign, int astride, int col, float lambda,
                              const int32_t* __restrict__ cand) {
  int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (p >= n) return;
  int cid[2] = {cand[p * 2], cand[p * 2 + 1]};
  float rn2[kMaxDirs];
  float loss[2] = {0.f, 0.f};
  // squared norms of the earlier residuals
  for (int r = 0; r < col; ++r) {
    const float* cr = C + (int64_t)assign[p * astride + r] * d;
    float s = 0.f;
    for (int k = lane; k < d; k += 32) {
      float v = load_elem(X, p * d + k) - cr[k];
      s = fmaf(v, v, s);
    }
    rn2[r] = warp_sum(s);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (cid[q] < 0) { loss[q] = INFINITY; continue; }
    const float* cq = C + (int64_t)cid[q] * d;
    float dist = 0.f;
    for (int k = lane; k < d; k += 32) {
      float v = load_elem(X, p * d + k) - cq[k];
      dist = fmaf(v, v, dist);
    }
    dist = warp_sum(dist);
    float pen = 0.f;
    for (int r = 0; r < col; ++r) {
      if (!(rn2[r] > 0.f)) continue;
      const float* cr = C + (int64_t)assign[p * astride + r] * d;
      float pr = 0.f;
      for (int k = lane; k < d; k += 32) {
        float xv = load_elem(X, p * d + k);
        pr = fmaf(xv - cq[k], xv - cr[k], pr);
      }
      pr = warp_sum(pr);
      pen += pr * pr / rn2[r];
    }
    loss[q] = fmaf(lambda, pen, dist);
  }
  if (lane == 0) {
    bool second = cid[1] >= 0 && (loss[1] < loss[0] || (loss[1] == loss[0] && cid[1] < cid[0]));
    assign[p * astride + col] = second ? cid[1] : cid[0];
  }
}

template <typename XT>
void screen_launch(int ndir, const XT* X, int64_t n, int d, const float* C, const float* cnorm, int c,
                   const int32_t* assign, int astride, const float* inv_rn, const float* xr,
                   float lambda, int32_t* cand, cudaStream_t s) {
  dim3 grid(ceil_div(n, BM));
  switch (ndir) {
    case 0: screen_kernel<0, XT><<<grid, kThreads, 0, s>>>(X, n, d, C, cnorm, c, assign, astride, inv_rn, xr, lambda, cand); break;
    case 1: screen_kernel<1, XT><<<grid, kThreads, 0, s>>>(X, n, d, C, cnorm, c, assign, astride, inv_rn, xr, lambda, cand); break;
    case 2: screen_kernel<2, XT><<<grid, kThreads, 0, s>>>(X, n, d, C, cnorm, c, assign, astride, inv_rn, xr, lambda, cand); break;
    case 3: screen_kernel<3, XT><<<grid, kThreads, 0, s>>>(X, n, d, C, cnorm, c, assign, astride, inv_rn, xr, lambda, cand); break;
    case 4: screen_kernel<4, XT><<<grid, kThreads, 0, s>>>(X, n, d, C, cnorm, c, assign, astride, inv_rn, xr, lambda, cand); break;
    default: fail(SOAR_EUNSUPPORTED, "screen: more than 4 residual directions");
  }
  SOAR_LAUNCHED();
}

template <typename XT>
void assign_typed(const XT* X, int64_t n, int32_t d, const float* C, int32_t c, float lambda,
                  int32_t spills, int32_t* assign, cudaStream_t s, Scratch& scr) {
  const int astride = 1 + spills;
  float* cnorm = scr.get<float>(c);
  int32_t* cand = scr.get<int32_t>((size_t)n * 2);
  float* inv_rn = nullptr;
  float* xr = nullptr;
  if (spills > 0) {
    inv_rn = scr.get<float>((size_t)n * kMaxDirs);
    xr = scr.get<float>((size_t)n * kMaxDirs);
  }
  centroid_norms<<<ceil_div((int64_t)c * 32, 256), 256, 0, s>>>(C, c, d, cnorm);
  SOAR_LAUNCHED();
  const unsigned wgrid = ceil_div(n * 32, 256);
  for (int j = 0; j <= spills; ++j) {
    if (j > 0) {
      residual_kernel<XT><<<wgrid, 256, 0, s>>>(X, n, d, C, assign, astride, j - 1, inv_rn, xr);
      SOAR_LAUNCHED();
    }
    if (assign_tc_supported(d, j)) {
      // primary and first spill: tensor-core screen with rigorous bounds
      assign_tc_pass<XT>(X, n, d, C, c, j, assign, astride, inv_rn, lambda, s, scr);
      continue;
    }
    screen_launch<XT>(j, X, n, d, C, cnorm, c, assign, astride, inv_rn, xr, lambda, cand, s);
    refine_kernel<XT><<<wgrid, 256, 0, s>>>(X, n, d, C, assign, astride, j, lambda, cand);
    SOAR_LAUNCHED();
  }
}

// ---------------------------------------------------------------- k-means

__global__ void iota_keys(const int32_t* assign, int64_t n, uint32_t* keys, int32_t* vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = (uint32_t)assign[i];
  vals[i] = (int32_t)i;
}

__global__ void check_indices(const int32_t* idx, int c, int64_t n, int* bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < c && (idx[i] < 0 || idx[i] >= n)) atomicOr(bad, 1);
}

template <typename XT>
__global__ void gather_rows_f32(const XT* __restrict__ X, int d, const int32_t* __restrict__ idx, int c,
                                float* __restrict__ C) {
  int r = blockIdx.x;
  if (r >= c) return;
  for (int k = threadIdx.x; k < d; k += blockDim.x) C[(int64_t)r * d + k] = load_elem(X, (int64_t)idx[r] * d + k);
}

// Centroid update: fp64 sum of each cluster's members (in ascending point
// order, four interleaved partial sums combined in a fixed order), mean
// rounded to fp32; empty clusters keep their centroid.
template <typename XT>
__global__ void kmeans_update(const XT* __restrict__ X, int d, const int32_t* __restrict__ members,
                              const int64_t* __restrict__ offsets, float* __restrict__ C) {
  const int p = blockIdx.x;
  const int64_t b = offsets[p], e = offsets[p + 1];
  const int64_t cnt = e - b;
  if (cnt == 0) return;
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    int64_t i = b;
    for (; i + 4 <= e; i += 4) {
      s0 += (double)load_elem(X, (int64_t)members[i] * d + k);
      s1 += (double)load_elem(X, (int64_t)members[i + 1] * d + k);
      s2 += (double)load_elem(X, (int64_t)members[i + 2] * d + k);
      s3 += (double)load_elem(X, (int64_t)members[i + 3] * d + k);
    }
    for (; i < e; ++i) s0 += (double)load_elem(X, (int64_t)members[i] * d + k);
    double sum = (s0 + s1) + (s2 + s3);
    C[(int64_t)p * d + k] = (float)(sum / (double)cnt);
  }
}

template <typename XT>
void kmeans_typed(const XT* X, int64_t n, int32_t d, int32_t c, int32_t iters, const int32_t* init_idx,
                  float* C, cudaStream_t s, Scratch& scr) {
  // the seed rows are caller input: reject indices outside [0, n) before using them
  int* bad = scr.get<int>(1);
  SOAR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  check_indices<<<ceil_div(c, 256), 256, 0, s>>>(init_idx, c, n, bad);
  SOAR_LAUNCHED();
  int hbad = 0;
  SOAR_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  SOAR_CUDA(cudaStreamSynchronize(s));
  if (hbad) fail(SOAR_EINVAL, "soar_train_centroids: init_idx entries must lie in [0, n)");
  gather_rows_f32<XT><<<c, 128, 0, s>>>(X, d, init_idx, c, C);
  SOAR_LAUNCHED();
  if (iters == 0) return;
  int32_t* assign = scr.get<int32_t>(n);
  uint32_t* keys = scr.get<uint32_t>(n);
  int32_t* vals = scr.get<int32_t>(n);
  uint32_t* keys2 = scr.get<uint32_t>(n);
  int32_t* vals2 = scr.get<int32_t>(n);
  int64_t* offsets = scr.get<int64_t>((size_t)c + 1);
  const int bits = bits_for(c);
  for (int it = 0; it < iters; ++it) {
    assign_typed<XT>(X, n, d, C, c, 0.f, 0, assign, s, scr);
    iota_keys<<<ceil_div(n, 256), 256, 0, s>>>(assign, n, keys, vals);
    SOAR_LAUNCHED();
    bool in_tmp = radix_sort_pairs(keys, vals, keys2, vals2, n, bits, s, scr);
    const uint32_t* ks = in_tmp ? keys2 : keys;
    const int32_t* vs = in_tmp ? vals2 : vals;
    segment_offsets(ks, n, c, offsets, s);
    kmeans_update<XT><<<c, 128, 0, s>>>(X, d, vs, offsets, C);
    SOAR_LAUNCHED();
  }
}

}  // namespace

void assign_points(const void* X, soar_dtype dt, int64_t n, int32_t d, const float* C, int32_t c,
                   float lambda, int32_t spills, int32_t* assign, cudaStream_t s, Scratch& scr) {
  if (spills > kMaxDirs) fail(SOAR_EUNSUPPORTED, "soar_assign: at most 4 spills");
  if (dt == SOAR_F32)
    assign_typed<float>(static_cast<const float*>(X), n, d, C, c, lambda, spills, assign, s, scr);
  else
    assign_typed<__nv_bfloat16>(static_cast<const __nv_bfloat16*>(X), n, d, C, c, lambda, spills, assign, s, scr);
}

void kmeans_train(const void* X, soar_dtype dt, int64_t n, int32_t d, int32_t c, int32_t iters,
                  const int32_t* init_idx, float* C, cudaStream_t s, Scratch& scr) {
  if (dt == SOAR_F32)
    kmeans_typed<float>(static_cast<const float*>(X), n, d, c, iters, init_idx, C, s, scr);
  else
    kmeans_typed<__nv_bfloat16>(static_cast<const __nv_bfloat16*>(X), n, d, c, iters, init_idx, C, s, scr);
}

}  // namespace soar
