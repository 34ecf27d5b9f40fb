// Learned probe count (not part of the paper): per-query features, labels,
// and a small MLP with its own forward, backward and Adam kernels.
//
// Features z(q) = [q || its top-64 centroid scores <q, C_i>, descending].
// Label t*(q) = the smallest probe count whose recall@k reaches the target:
// a true neighbour v is found at probe count t exactly when one of v's
// partitions sits at probe position <= t, so t* is the ceil(target k)-th
// smallest of those positions (position = 1 + #centroids ranked before p,
// ties to the lower id).
// Network: y = w3 . relu(W2 relu(W1 z + b1) + b2) + b3, trained by mean
// squared error against log t*; t(q) = clamp(ceil(alpha exp(y)), 1, c).
//
// Parameters live in one fp32 buffer: W1 [H][D] | b1 [H] | W2 [H][H] | b2 [H]
// | W3 [H] | b3 [1].  In bf16 mode the weights and inputs of every product
// are rounded to bf16 (round to nearest even) and products accumulate in fp32;
// the fp32 master weights take the Adam updates.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace soar {

namespace {

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// C[m][n] = op(sum_k A(m, k) B(k, n)) with strided operands:
//   A(m, k) = A[m * am + k * ak], B(k, n) = B[k * bk + n * bn]
// epilogue: + bias[n] (optional), relu (optional), times 1[G[m][n] > 0]
// (optional gate), bf16 rounding of the operands when round != 0.
__global__ void __launch_bounds__(256) gemm_strided(const float* __restrict__ A, int64_t am, int64_t ak,
                                                    const float* __restrict__ B, int64_t bk, int64_t bn,
                                                    float* __restrict__ C, int M, int N, int K,
                                                    const float* __restrict__ bias, int relu,
                                                    const float* __restrict__ gate, int round) {
  __shared__ float As[16][65];
  __shared__ float Bs[16][65];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int i = tid; i < 64 * 16; i += 256) {
      const int r = i / 16, kk = i % 16, k = k0 + kk;
      float a = (m0 + r < M && k < K) ? A[(int64_t)(m0 + r) * am + (int64_t)k * ak] : 0.f;
      float b = (n0 + r < N && k < K) ? B[(int64_t)k * bk + (int64_t)(n0 + r) * bn] : 0.f;
      if (round) { a = bf16r(a); b = bf16r(b); }
      As[kk][r] = a;
      Bs[kk][r] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (bias) v += bias[n];
      if (relu) v = fmaxf(v, 0.f);
      if (gate && !(gate[(int64_t)m * N + n] > 0.f)) v = 0.f;
      C[(int64_t)m * N + n] = v;
    }
  }
}

// out[n] = sum over m of X[m][n] (fixed order per column), times `scale`.
__global__ void column_sums(const float* __restrict__ X, int M, int N, float scale, float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += X[(int64_t)m * N + n];
  out[n] = s * scale;
}

// gy[m] = 2 (y[m] - target[m]) / B and the loss mean((y - target)^2) (one block).
__global__ void mse_grad(const float* __restrict__ y, const float* __restrict__ target, int B, float* __restrict__ gy,
                         float* __restrict__ loss) {
  __shared__ float red[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    const float e = y[i] - target[i];
    gy[i] = 2.f * e / (float)B;
    s += e * e;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = red[0] / (float)B;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, int64_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.f - b1) * gi;
  const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

__global__ void probes_from_output(const float* __restrict__ y, int B, float alpha, int c, int32_t* __restrict__ t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const float v = ceilf(alpha * expf(y[i]));
  t[i] = (int32_t)fminf(fmaxf(v, 1.f), (float)c);
}

// Features: [q || top-`top` centroid scores, descending] (top list from top-t).
template <typename QT>
__global__ void build_features(const QT* __restrict__ Q, int64_t nq, int d, const float* __restrict__ top_s, int top,
                               float* __restrict__ Z) {
  const int64_t q = blockIdx.x;
  const int D = d + top;
  for (int i = threadIdx.x; i < D; i += blockDim.x)
    Z[q * D + i] = i < d ? load_elem(Q, q * d + i) : top_s[q * top + (i - d)];
}

// Label kernel: block per query.  Position of partition p in the query's
// probe order = 1 + #{i : s_i > s_p or (s_i == s_p and i < p)}.
__global__ void label_kernel(const float* __restrict__ S, int c, const int64_t* __restrict__ truth, int k,
                             const int32_t* __restrict__ assign, int a, int64_t n, int need,
                             int32_t* __restrict__ labels) {
  extern __shared__ int32_t posv[];   // [k]
  const int64_t q = blockIdx.x;
  const float* row = S + q * c;
  __shared__ int32_t red[32];
  for (int v = 0; v < k; ++v) {
    const int64_t id = truth[q * k + v];
    int best = 0x7fffffff;           // an id outside [0, n) is never found
    if (id >= 0 && id < n) {
      for (int j = 0; j < a; ++j) {
        const int p = assign[id * a + j];
        const float sp = row[p];
        int cnt = 0;
        for (int i = threadIdx.x; i < c; i += blockDim.x) {
          const float si = row[i];
          cnt += (si > sp) || (si == sp && i < p);
        }
        cnt = warp_sum(cnt);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
          int tot = 0;
          for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
          best = min(best, tot + 1);
        }
        __syncthreads();
      }
    }
    if (threadIdx.x == 0) posv[v] = best;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // need-th smallest position (insertion sort of k values)
    for (int i = 1; i < k; ++i) {
      const int x = posv[i];
      int j = i - 1;
      while (j >= 0 && posv[j] > x) { posv[j + 1] = posv[j]; --j; }
      posv[j + 1] = x;
    }
    labels[q] = posv[need - 1];
  }
}

inline void gemm(const float* A, int64_t am, int64_t ak, const float* B, int64_t bk, int64_t bn, float* C, int M,
                 int N, int K, const float* bias, bool relu, const float* gate, bool round, cudaStream_t s) {
  dim3 grid(ceil_div(N, 64), ceil_div(M, 64));
  gemm_strided<<<grid, 256, 0, s>>>(A, am, ak, B, bk, bn, C, M, N, K, bias, relu ? 1 : 0, gate, round ? 1 : 0);
  SOAR_LAUNCHED();
}

struct Layout {
  int64_t W1, b1, W2, b2, W3, b3, total;
  Layout(int D, int H) {
    W1 = 0;
    b1 = W1 + (int64_t)H * D;
    W2 = b1 + H;
    b2 = W2 + (int64_t)H * H;
    W3 = b2 + H;
    b3 = W3 + H;
    total = b3 + 1;
  }
};

}  // namespace

int64_t mlp_param_count(int D, int H) { return Layout(D, H).total; }

// Forward into caller-provided activations (A1, H1, A2, H2 of [B][H], y [B]).
void mlp_forward(const float* P, int D, int H, const float* Z, int B, bool bf16, float* A1, float* H1, float* A2,
                 float* H2, float* y, cudaStream_t s) {
  const Layout L(D, H);
  // A1 = Z W1^T + b1 ; H1 = relu(A1)
  gemm(Z, D, 1, P + L.W1, 1, D, A1, B, H, D, P + L.b1, false, nullptr, bf16, s);
  gemm(Z, D, 1, P + L.W1, 1, D, H1, B, H, D, P + L.b1, true, nullptr, bf16, s);
  gemm(H1, H, 1, P + L.W2, 1, H, A2, B, H, H, P + L.b2, false, nullptr, bf16, s);
  gemm(H1, H, 1, P + L.W2, 1, H, H2, B, H, H, P + L.b2, true, nullptr, bf16, s);
  gemm(H2, H, 1, P + L.W3, 1, 0, y, B, 1, H, P + L.b3, false, nullptr, bf16, s);
}

void mlp_backward(const float* P, int D, int H, const float* Z, const float* target, int B, bool bf16, float* G,
                  float* loss, cudaStream_t s, Scratch& scr) {
  const Layout L(D, H);
  float* A1 = scr.get<float>((size_t)B * H);
  float* H1 = scr.get<float>((size_t)B * H);
  float* A2 = scr.get<float>((size_t)B * H);
  float* H2 = scr.get<float>((size_t)B * H);
  float* y = scr.get<float>(B);
  float* gy = scr.get<float>(B);
  float* gA2 = scr.get<float>((size_t)B * H);
  float* gA1 = scr.get<float>((size_t)B * H);
  mlp_forward(P, D, H, Z, B, bf16, A1, H1, A2, H2, y, s);
  mse_grad<<<1, 256, 0, s>>>(y, target, B, gy, loss);
  SOAR_LAUNCHED();
  // gW3[h] = sum_b gy[b] H2[b][h]; gb3 = sum gy
  gemm(gy, 0, 1, H2, H, 1, G + L.W3, 1, H, B, nullptr, false, nullptr, bf16, s);
  column_sums<<<1, 32, 0, s>>>(gy, B, 1, 1.f, G + L.b3);
  SOAR_LAUNCHED();
  // gA2[b][h] = gy[b] W3[h] * 1[A2 > 0]
  gemm(gy, 1, 0, P + L.W3, 0, 1, gA2, B, H, 1, nullptr, false, A2, bf16, s);
  // gW2 = gA2^T H1 ; gb2 = colsum(gA2)
  gemm(gA2, 1, H, H1, H, 1, G + L.W2, H, H, B, nullptr, false, nullptr, bf16, s);
  column_sums<<<ceil_div(H, 128), 128, 0, s>>>(gA2, B, H, 1.f, G + L.b2);
  SOAR_LAUNCHED();
  // gA1 = (gA2 W2) * 1[A1 > 0]
  gemm(gA2, H, 1, P + L.W2, H, 1, gA1, B, H, H, nullptr, false, A1, bf16, s);
  // gW1 = gA1^T Z ; gb1 = colsum(gA1)
  gemm(gA1, 1, H, Z, D, 1, G + L.W1, H, D, B, nullptr, false, nullptr, bf16, s);
  column_sums<<<ceil_div(H, 128), 128, 0, s>>>(gA1, B, H, 1.f, G + L.b1);
  SOAR_LAUNCHED();
}

void mlp_adam(float* P, const float* G, float* m1, float* m2, int64_t n, int step, float lr, float b1, float b2,
              float eps, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<ceil_div(n, 256), 256, 0, s>>>(P, G, m1, m2, n, lr, b1, b2, eps, c1, c2);
  SOAR_LAUNCHED();
}

void mlp_predict(const float* P, int D, int H, const float* Z, int B, bool bf16, float alpha, int c, float* y_out,
                 int32_t* t_out, cudaStream_t s, Scratch& scr) {
  float* A1 = scr.get<float>((size_t)B * H);
  float* H1 = scr.get<float>((size_t)B * H);
  float* A2 = scr.get<float>((size_t)B * H);
  float* H2 = scr.get<float>((size_t)B * H);
  float* y = y_out ? y_out : scr.get<float>(B);
  mlp_forward(P, D, H, Z, B, bf16, A1, H1, A2, H2, y, s);
  if (t_out) {
    probes_from_output<<<ceil_div(B, 256), 256, 0, s>>>(y, B, alpha, c, t_out);
    SOAR_LAUNCHED();
  }
}

void probe_features(const IndexData& ix, const void* Q, soar_dtype dt, int64_t nq, int top, float* Z,
                    cudaStream_t s, Scratch& scr) {
  int32_t* t_ids = scr.get<int32_t>((size_t)nq * top);
  float* t_s = scr.get<float>((size_t)nq * top);
  select_partitions(ix, Q, dt, nq, top, t_ids, t_s, s, scr);
  if (dt == SOAR_F32)
    build_features<float><<<(unsigned)nq, 128, 0, s>>>(static_cast<const float*>(Q), nq, ix.d, t_s, top, Z);
  else
    build_features<__nv_bfloat16><<<(unsigned)nq, 128, 0, s>>>(static_cast<const __nv_bfloat16*>(Q), nq, ix.d, t_s,
                                                               top, Z);
  SOAR_LAUNCHED();
}

void features_from_scores(const void* Q, soar_dtype dt, int64_t nq, int d, const float* top_s, int top, float* Z,
                          cudaStream_t s) {
  if (dt == SOAR_F32)
    build_features<float><<<(unsigned)nq, 128, 0, s>>>(static_cast<const float*>(Q), nq, d, top_s, top, Z);
  else
    build_features<__nv_bfloat16><<<(unsigned)nq, 128, 0, s>>>(static_cast<const __nv_bfloat16*>(Q), nq, d, top_s,
                                                               top, Z);
  SOAR_LAUNCHED();
}

void probe_labels(const IndexData& ix, const void* Q, soar_dtype dt, int64_t nq, const int64_t* truth, int k,
                  float target, int32_t* labels, cudaStream_t s, Scratch& scr) {
  // every centroid score of every query, computed exactly as the search ranks them
  float* S = scr.get<float>((size_t)nq * ix.c);
  centroid_scores(ix, Q, dt, nq, S, s, scr);
  const int need = std::max(1, (int)ceilf(target * (float)k - 1e-6f));
  label_kernel<<<(unsigned)nq, 256, sizeof(int32_t) * k, s>>>(S, ix.c, truth, k, ix.assign, 1 + ix.spills, ix.n,
                                                             std::min(need, k), labels);
  SOAR_LAUNCHED();
}

}  // namespace soar
