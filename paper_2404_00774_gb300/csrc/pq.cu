// 4-bit product quantization of the partitioning residuals (Section 3.5,
// App. A.3): each residual r = x - C_p is split into subspaces of two
// dimensions, each quantized to the nearest of 16 centres (a 4-bit code).
// Training: per-subspace Lloyd's k-means on the residuals of a sample, each
// centre the fp64 mean of its rows summed in a fixed order (deterministic),
// rounded to fp32.  Encoding: the code of every index row (every copy of a
// point) from its own residual, so a spilled point carries one code per
// partition it is assigned to.
#include "internal.cuh"

namespace soar {

namespace {

constexpr int kPqCentres = 16;

// Nearest of the 16 centres of one subspace (direct form in fp32, the lower
// index on ties).
__device__ __forceinline__ int pq_nearest(float r0, float r1, const float* __restrict__ Bs) {
  int best = 0;
  float bd = INFINITY;
#pragma unroll
  for (int j = 0; j < kPqCentres; ++j) {
    const float d0 = r0 - Bs[2 * j], d1 = r1 - Bs[2 * j + 1];
    const float dist = fmaf(d1, d1, d0 * d0);
    if (dist < bd) {
      bd = dist;
      best = j;
    }
  }
  return best;
}

// Residual rows R[i] = X[i] - C[part[i]] in fp32.
template <typename T>
__global__ void pq_residuals_kernel(const T* __restrict__ X, int64_t n, int d, const float* __restrict__ C,
                                    const int32_t* __restrict__ part, float* __restrict__ R) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * d) return;
  const int64_t i = e / d;
  const int k = (int)(e - i * d);
  R[e] = load_elem(X, e) - C[(int64_t)part[i] * d + k];
}

// B[s][j] = R[init[j]][2s .. 2s+1].
__global__ void pq_init_kernel(const float* __restrict__ R, int d, const int32_t* __restrict__ init, int m,
                               float* __restrict__ B) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * kPqCentres) return;
  const int s = e / kPqCentres, j = e % kPqCentres;
  B[2 * e] = R[(int64_t)init[j] * d + 2 * s];
  B[2 * e + 1] = R[(int64_t)init[j] * d + 2 * s + 1];
}

// code[i][s] of every training row.
__global__ void pq_assign_kernel(const float* __restrict__ R, int64_t n, int d, int m, const float* __restrict__ B,
                                 uint8_t* __restrict__ code) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m) return;
  const int64_t i = e / m;
  const int s = (int)(e - i * m);
  code[e] = (uint8_t)pq_nearest(R[i * d + 2 * s], R[i * d + 2 * s + 1], B + (size_t)s * 2 * kPqCentres);
}

// A block per (subspace, centre): the fp64 sums of its rows, each thread
// over a fixed stride of rows, then a fixed-order tree reduction, so the
// result does not depend on scheduling; the new centre is the mean rounded
// to fp32, an empty centre keeps its value.
constexpr int kUpdThreads = 256;
__global__ void __launch_bounds__(kUpdThreads) pq_update_kernel(const float* __restrict__ R, int64_t n, int d, int m,
                                                                const uint8_t* __restrict__ code,
                                                                float* __restrict__ B) {
  __shared__ double s0[kUpdThreads], s1[kUpdThreads];
  __shared__ long long cnt_s[kUpdThreads];
  const int s = blockIdx.x / kPqCentres, j = blockIdx.x % kPqCentres;
  double a0 = 0.0, a1 = 0.0;
  long long cnt = 0;
  for (int64_t i = threadIdx.x; i < n; i += kUpdThreads) {
    if (code[i * m + s] != j) continue;
    a0 += (double)R[i * d + 2 * s];
    a1 += (double)R[i * d + 2 * s + 1];
    ++cnt;
  }
  s0[threadIdx.x] = a0;
  s1[threadIdx.x] = a1;
  cnt_s[threadIdx.x] = cnt;
  __syncthreads();
  for (int h = kUpdThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s0[threadIdx.x] += s0[threadIdx.x + h];
      s1[threadIdx.x] += s1[threadIdx.x + h];
      cnt_s[threadIdx.x] += cnt_s[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && cnt_s[0] > 0) {
    const size_t o = ((size_t)s * kPqCentres + j) * 2;
    B[o] = (float)(s0[0] / (double)cnt_s[0]);
    B[o + 1] = (float)(s1[0] / (double)cnt_s[0]);
  }
}

// Partition of every index row (the rows of p are offsets[p] .. offsets[p+1]).
__global__ void row_partitions(const int64_t* __restrict__ off, int c, int32_t* __restrict__ part) {
  const int p = blockIdx.x;
  if (p >= c) return;
  for (int64_t r = off[p] + threadIdx.x; r < off[p + 1]; r += blockDim.x) part[r] = p;
}

// A thread per (index row, code byte): subspaces 2b (low nibble) and 2b + 1
// (high nibble) of the row's residual x - C_p; bytes past the codes are 0.
template <typename T>
__global__ void pq_encode_kernel(const T* __restrict__ X, int d, const float* __restrict__ C,
                                 const int32_t* __restrict__ ids, const int32_t* __restrict__ part, int64_t rows,
                                 int m, const float* __restrict__ B, int code_stride, uint8_t* __restrict__ codes) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * code_stride) return;
  const int64_t r = e / code_stride;
  const int b = (int)(e - r * code_stride);
  uint8_t v = 0;
  const int64_t x0 = (int64_t)ids[r] * d;
  const int64_t c0 = (int64_t)part[r] * d;
  for (int h = 0; h < 2; ++h) {
    const int s = 2 * b + h;
    if (s >= m) break;
    const float r0 = load_elem(X, x0 + 2 * s) - C[c0 + 2 * s];
    const float r1 = load_elem(X, x0 + 2 * s + 1) - C[c0 + 2 * s + 1];
    v |= (uint8_t)(pq_nearest(r0, r1, B + (size_t)s * 2 * kPqCentres) << (4 * h));
  }
  codes[e] = v;
}

}  // namespace

void pq_train(const void* X, soar_dtype dt, int64_t n, int32_t d, const float* C, const int32_t* part,
              int32_t iters, const int32_t* init_idx, float* B, cudaStream_t s, Scratch& scr) {
  const int m = d / 2;
  float* R = scr.get<float>((size_t)n * d);
  uint8_t* code = scr.get<uint8_t>((size_t)n * m);
  if (dt == SOAR_F32)
    pq_residuals_kernel<float><<<ceil_div(n * d, 256), 256, 0, s>>>(static_cast<const float*>(X), n, d, C, part, R);
  else
    pq_residuals_kernel<__nv_bfloat16><<<ceil_div(n * d, 256), 256, 0, s>>>(static_cast<const __nv_bfloat16*>(X), n,
                                                                           d, C, part, R);
  SOAR_LAUNCHED();
  pq_init_kernel<<<ceil_div((int64_t)m * kPqCentres, 256), 256, 0, s>>>(R, d, init_idx, m, B);
  SOAR_LAUNCHED();
  for (int it = 0; it < iters; ++it) {
    pq_assign_kernel<<<ceil_div(n * m, 256), 256, 0, s>>>(R, n, d, m, B, code);
    SOAR_LAUNCHED();
    pq_update_kernel<<<m * kPqCentres, kUpdThreads, 0, s>>>(R, n, d, m, code, B);
    SOAR_LAUNCHED();
  }
}

void pq_encode_index(IndexData& ix, const void* X, soar_dtype dt, cudaStream_t s, Scratch& scr) {
  int32_t* part = scr.get<int32_t>(ix.rows);
  row_partitions<<<ix.c, 256, 0, s>>>(ix.offsets, ix.c, part);
  SOAR_LAUNCHED();
  const int64_t total = ix.rows * ix.code_stride;
  if (dt == SOAR_F32)
    pq_encode_kernel<float><<<ceil_div(total, 256), 256, 0, s>>>(static_cast<const float*>(X), ix.d, ix.centroids,
        ix.ids, part, ix.rows, ix.pq_m, ix.pq_cb, ix.code_stride, static_cast<uint8_t*>(ix.vectors));
  else
    pq_encode_kernel<__nv_bfloat16><<<ceil_div(total, 256), 256, 0, s>>>(static_cast<const __nv_bfloat16*>(X), ix.d,
        ix.centroids, ix.ids, part, ix.rows, ix.pq_m, ix.pq_cb, ix.code_stride, static_cast<uint8_t*>(ix.vectors));
  SOAR_LAUNCHED();
}

}  // namespace soar
