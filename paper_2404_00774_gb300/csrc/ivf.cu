// Inverted-file index build (Section 2.2) with spilled copies (Section 3.5).
//
// The n (1 + s) (partition, point) pairs are sorted by partition with a
// stable radix sort, so each partition lists its members in ascending point
// id.  Each member's vector is then copied next to its id: partition p is
// one contiguous block of rows, which is what the search streams.
#include <algorithm>

#include "internal.cuh"

namespace soar {

namespace {

__global__ void check_assign(const int32_t* assign, int64_t n, int a, int c, int* bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int j = 0; j < a; ++j) {
    int v = assign[i * a + j];
    if (v < 0 || v >= c) { atomicOr(bad, 1); return; }
    for (int jj = 0; jj < j; ++jj)
      if (assign[i * a + jj] == v) { atomicOr(bad, 2); return; }
  }
}

__global__ void pair_keys(const int32_t* assign, int64_t n, int a, uint32_t* keys, int32_t* vals) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * a) return;
  keys[e] = (uint32_t)assign[e];
  vals[e] = (int32_t)(e / a);
}

// rows[e][0..stride) = X[ids[e]][0..d) then zeros.
template <typename T>
__global__ void gather_rows(const T* __restrict__ X, int d, const int32_t* __restrict__ ids, int64_t rows,
                            int stride, T* __restrict__ out) {
  int64_t e = blockIdx.x;
  if (e >= rows) return;
  const T* src = X + (int64_t)(ids ? ids[e] : e) * d;
  T* dst = out + e * stride;
  for (int k = threadIdx.x; k < stride; k += blockDim.x) dst[k] = k < d ? src[k] : T(0.f);
}

// Warp per row: scale = max|v| / 448 (1 for a zero row); codes = e4m3(v / scale),
// round to nearest even, saturating at +-448.
template <typename T>
__global__ void quantize_rows(const T* __restrict__ V, int64_t m, int d, const int32_t* __restrict__ ids,
                              uint8_t* __restrict__ codes, int code_stride, float* __restrict__ scales) {
  int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (r >= m) return;
  const T* src = V + (int64_t)(ids ? ids[r] : r) * d;
  float amax = 0.f;
  for (int k = lane; k < d; k += 32) amax = fmaxf(amax, fabsf(load_elem(src, k)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const float scale = amax > 0.f ? amax / 448.f : 1.f;
  uint8_t* dst = codes + r * code_stride;
  for (int k = lane; k < code_stride; k += 32) {
    uint8_t q = 0;
    if (k < d) q = (uint8_t)__nv_cvt_float_to_fp8(load_elem(src, k) / scale, __NV_SATFINITE, __NV_E4M3);
    dst[k] = q;
  }
  if (lane == 0) scales[r] = scale;
}

__global__ void decode_codes(const uint8_t* __restrict__ codes, int64_t count, float* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)codes[i], __NV_E4M3);
  out[i] = __half2float(__half(h));
}

// key = largest size - size (so an ascending stable sort puts big partitions first)
__global__ void size_keys(const int64_t* __restrict__ off, int c, int64_t mx, uint32_t* __restrict__ keys,
                          int32_t* __restrict__ vals) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= c) return;
  keys[p] = (uint32_t)(mx - (off[p + 1] - off[p]));
  vals[p] = p;
}

__global__ void group_counts(const int64_t* __restrict__ off, int c, int64_t* __restrict__ cnt) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > c) return;
  cnt[p] = p < c ? (off[p + 1] - off[p] + 7) / 8 : 0;
}

// Partition p's rows -> 8-row groups in the core-matrix layout (tc.cuh): with
// E = 16 / sizeof(T) elements per 16-byte row chunk, element k of padded row
// i goes to group gstart[p] + i/8, element (k/E)*8E + (i%8)*E + k%E.
template <typename T>
__global__ void fill_tc_rows(const T* __restrict__ rows, int row_stride, int d, const int64_t* __restrict__ off,
                             const int32_t* __restrict__ ids, const int64_t* __restrict__ gstart, int kp,
                             T* __restrict__ out, int32_t* __restrict__ out_ids) {
  constexpr int E = 16 / (int)sizeof(T);
  const int p = blockIdx.x;
  const int64_t r0 = off[p];
  const int size = (int)(off[p + 1] - r0);
  const int64_t g0 = gstart[p];
  const int padded = (int)(gstart[p + 1] - g0) * 8;
  for (int64_t idx = threadIdx.x; idx < (int64_t)padded * kp; idx += blockDim.x) {
    const int i = (int)(idx / kp), k = (int)(idx % kp);
    const T v = (i < size && k < d) ? rows[(r0 + i) * row_stride + k] : T(0.f);
    out[(g0 + i / 8) * (int64_t)(8 * kp) + (k / E) * (8 * E) + (i % 8) * E + (k % E)] = v;
  }
  for (int i = threadIdx.x; i < padded; i += blockDim.x) out_ids[g0 * 8 + i] = i < size ? ids[r0 + i] : -1;
}

// ||x|| of every padded row (warp per row).
template <typename T>
__global__ void tc_row_norms(const T* __restrict__ tc_rows, int64_t nrows_padded, int kp, float* __restrict__ norms) {
  constexpr int E = 16 / (int)sizeof(T);
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= nrows_padded) return;
  const T* g = tc_rows + (r / 8) * (int64_t)(8 * kp) + (r % 8) * E;
  float acc = 0.f;
  for (int k = lane; k < kp; k += 32) {
    const float v = load_elem(g, (k / E) * (8 * E) + (k % E));
    acc = fmaf(v, v, acc);
  }
  acc = warp_sum(acc);
  if (lane == 0) norms[r] = sqrtf(acc);
}

// Largest row norm of every partition (block per partition).
__global__ void partition_max_norm(const float* __restrict__ norms, const int64_t* __restrict__ gstart,
                                   float* __restrict__ pmax) {
  const int p = blockIdx.x;
  float mx = 0.f;
  for (int64_t r = gstart[p] * 8 + threadIdx.x; r < gstart[p + 1] * 8; r += blockDim.x) mx = fmaxf(mx, norms[r]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ float wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, wm[w]);
    pmax[p] = mx;
  }
}

__global__ void chunk_offsets(int64_t n, int64_t chunk, int c, int64_t* __restrict__ off,
                              int64_t* __restrict__ gstart, int32_t* __restrict__ order) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > c) return;
  const int64_t r = min(n, (int64_t)p * chunk);
  off[p] = r;
  gstart[p] = (int64_t)p * (chunk / 8);     // every chunk but the last is a whole number of groups
  if (p < c) order[p] = p;
}

__global__ void iota_i32(int32_t* __restrict__ a, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = (int32_t)i;
}

}  // namespace

void build_flat_tc(IndexData& fx, int64_t chunk, cudaStream_t s, Scratch& scr) {
  const int64_t n = fx.n;
  const int c = fx.c, d = fx.d;
  const size_t esz = fx.dtype == SOAR_F32 ? 4 : 2;
  const int kstep = fx.dtype == SOAR_F32 ? 8 : 16;
  fx.tc_kp = (d + kstep - 1) / kstep * kstep;
  fx.offsets = scr.get<int64_t>((size_t)c + 1);
  fx.tc_gstart = scr.get<int64_t>((size_t)c + 1);
  fx.part_order = scr.get<int32_t>(c);
  chunk_offsets<<<ceil_div((int64_t)c + 1, 256), 256, 0, s>>>(n, chunk, c, fx.offsets, fx.tc_gstart, fx.part_order);
  SOAR_LAUNCHED();
  // the last chunk's group count: its rows rounded up to 8
  const int64_t groups = (int64_t)(c - 1) * (chunk / 8) + (n - (int64_t)(c - 1) * chunk + 7) / 8;
  fx.tc_groups = groups;
  SOAR_CUDA(cudaMemcpyAsync(fx.tc_gstart + c, &groups, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  SOAR_CUDA(cudaStreamSynchronize(s));   // the host value above must not go out of scope before the copy
  fx.ids = scr.get<int32_t>(n);
  iota_i32<<<ceil_div(n, 256), 256, 0, s>>>(fx.ids, n);
  SOAR_LAUNCHED();
  fx.tc_rows = scr.get<unsigned char>(esz * (size_t)groups * 8 * fx.tc_kp);
  fx.tc_ids = scr.get<int32_t>((size_t)groups * 8);
  fx.tc_norms = scr.get<float>((size_t)groups * 8);
  fx.tc_pmax = scr.get<float>(c);
  if (fx.dtype == SOAR_F32) {
    fill_tc_rows<float><<<c, 1024, 0, s>>>(static_cast<const float*>(fx.vectors), fx.row_stride, d, fx.offsets, fx.ids,
                                          fx.tc_gstart, fx.tc_kp, static_cast<float*>(fx.tc_rows), fx.tc_ids);
    SOAR_LAUNCHED();
    tc_row_norms<float><<<ceil_div(groups * 8 * 32, 256), 256, 0, s>>>(static_cast<const float*>(fx.tc_rows),
                                                                       groups * 8, fx.tc_kp, fx.tc_norms);
  } else {
    fill_tc_rows<__nv_bfloat16><<<c, 1024, 0, s>>>(static_cast<const __nv_bfloat16*>(fx.vectors), fx.row_stride, d,
                                                   fx.offsets, fx.ids, fx.tc_gstart, fx.tc_kp,
                                                  static_cast<__nv_bfloat16*>(fx.tc_rows), fx.tc_ids);
    SOAR_LAUNCHED();
    tc_row_norms<__nv_bfloat16><<<ceil_div(groups * 8 * 32, 256), 256, 0, s>>>(
        static_cast<const __nv_bfloat16*>(fx.tc_rows), groups * 8, fx.tc_kp, fx.tc_norms);
  }
  SOAR_LAUNCHED();
  partition_max_norm<<<c, 256, 0, s>>>(fx.tc_norms, fx.tc_gstart, fx.tc_pmax);
  SOAR_LAUNCHED();
}

void quantize_fp8(const void* V, soar_dtype dt, int64_t m, int32_t d, uint8_t* codes, int32_t code_stride,
                  float* scales, cudaStream_t s) {
  if (m == 0) return;
  unsigned grid = ceil_div(m * 32, 256);
  if (dt == SOAR_F32)
    quantize_rows<float><<<grid, 256, 0, s>>>(static_cast<const float*>(V), m, d, nullptr, codes, code_stride, scales);
  else
    quantize_rows<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(V), m, d, nullptr, codes,
                                                      code_stride, scales);
  SOAR_LAUNCHED();
}

// Builds every device array of the index; synchronises `s` once to read the
// validity flag and the partition sizes.
void build_index(IndexData& ix, const void* X, soar_dtype dt, const float* C, const int32_t* assign,
                 cudaStream_t s, const float* pq_cb) {
  Scratch scr(s);
  const int a = 1 + ix.spills;
  const int64_t n = ix.n, rows = ix.rows;
  const int d = ix.d, c = ix.c;
  const size_t esz = dt == SOAR_F32 ? 4 : 2;
  int* bad = scr.get<int>(1);
  SOAR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  check_assign<<<ceil_div(n, 256), 256, 0, s>>>(assign, n, a, c, bad);
  SOAR_LAUNCHED();

  auto dev_alloc = [&](void** p, size_t bytes) {
    SOAR_CUDA(cudaMalloc(p, bytes ? bytes : 16));
    ix.bytes += (int64_t)bytes;
  };
  dev_alloc((void**)&ix.offsets, sizeof(int64_t) * (c + 1));
  dev_alloc((void**)&ix.ids, sizeof(int32_t) * rows);
  dev_alloc((void**)&ix.centroids, sizeof(float) * (size_t)c * d);
  SOAR_CUDA(cudaMemcpyAsync(ix.centroids, C, sizeof(float) * (size_t)c * d, cudaMemcpyDeviceToDevice, s));
  dev_alloc((void**)&ix.assign, sizeof(int32_t) * (size_t)n * a);
  SOAR_CUDA(cudaMemcpyAsync(ix.assign, assign, sizeof(int32_t) * (size_t)n * a, cudaMemcpyDeviceToDevice, s));

  uint32_t* keys = scr.get<uint32_t>(rows);
  int32_t* vals = scr.get<int32_t>(rows);
  uint32_t* keys2 = scr.get<uint32_t>(rows);
  int32_t* vals2 = scr.get<int32_t>(rows);
  pair_keys<<<ceil_div(rows, 256), 256, 0, s>>>(assign, n, a, keys, vals);
  SOAR_LAUNCHED();
  bool in_tmp = radix_sort_pairs(keys, vals, keys2, vals2, rows, bits_for(c), s, scr);
  const uint32_t* ks = in_tmp ? keys2 : keys;
  const int32_t* vs = in_tmp ? vals2 : vals;
  segment_offsets(ks, rows, c, ix.offsets, s);
  SOAR_CUDA(cudaMemcpyAsync(ix.ids, vs, sizeof(int32_t) * rows, cudaMemcpyDeviceToDevice, s));

  // vector rows, 16-byte aligned
  if (ix.mode == SOAR_SCORE_F32) {
    ix.row_stride = (int)(((d * esz + 15) / 16) * 16 / esz);
    dev_alloc(&ix.vectors, esz * (size_t)rows * ix.row_stride);
    if (dt == SOAR_F32)
      gather_rows<float><<<(unsigned)rows, 128, 0, s>>>(static_cast<const float*>(X), d, vs, rows, ix.row_stride,
                                                        static_cast<float*>(ix.vectors));
    else
      gather_rows<__nv_bfloat16><<<(unsigned)rows, 128, 0, s>>>(static_cast<const __nv_bfloat16*>(X), d, vs, rows,
                                                                ix.row_stride, static_cast<__nv_bfloat16*>(ix.vectors));
    SOAR_LAUNCHED();
  } else if (ix.mode == SOAR_SCORE_FP8) {
    ix.code_stride = (d + 15) / 16 * 16;
    ix.row_stride = ix.code_stride;
    dev_alloc(&ix.vectors, (size_t)rows * ix.code_stride);
    dev_alloc((void**)&ix.row_scales, sizeof(float) * rows);
    const int ostride = (int)(((d * esz + 15) / 16) * 16 / esz);
    dev_alloc(&ix.originals, esz * (size_t)n * ostride);
    dev_alloc((void**)&ix.cent_scales, sizeof(float) * c);
    uint8_t* ccodes = scr.get<uint8_t>((size_t)c * ix.code_stride);
    dev_alloc((void**)&ix.cent_code_vals, sizeof(float) * (size_t)c * ix.code_stride);
    unsigned wg = ceil_div(rows * 32, 256);
    if (dt == SOAR_F32) {
      quantize_rows<float><<<wg, 256, 0, s>>>(static_cast<const float*>(X), rows, d, vs,
                                              static_cast<uint8_t*>(ix.vectors), ix.code_stride, ix.row_scales);
      gather_rows<float><<<(unsigned)n, 128, 0, s>>>(static_cast<const float*>(X), d, nullptr, n, ostride,
                                                     static_cast<float*>(ix.originals));
    } else {
      quantize_rows<__nv_bfloat16><<<wg, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(X), rows, d, vs,
                                                      static_cast<uint8_t*>(ix.vectors), ix.code_stride,
                                                      ix.row_scales);
      gather_rows<__nv_bfloat16><<<(unsigned)n, 128, 0, s>>>(static_cast<const __nv_bfloat16*>(X), d, nullptr, n,
                                                             ostride, static_cast<__nv_bfloat16*>(ix.originals));
    }
    SOAR_LAUNCHED();
    quantize_rows<float><<<ceil_div((int64_t)c * 32, 256), 256, 0, s>>>(ix.centroids, c, d, nullptr, ccodes,
                                                                        ix.code_stride, ix.cent_scales);
    SOAR_LAUNCHED();
    decode_codes<<<ceil_div((int64_t)c * ix.code_stride, 256), 256, 0, s>>>(ccodes, (int64_t)c * ix.code_stride,
                                                                          ix.cent_code_vals);
    SOAR_LAUNCHED();
  } else if (ix.mode == SOAR_SCORE_PQ4) {
    // two 4-bit codes per byte, rows padded to 16 bytes; the originals once
    ix.pq_m = d / 2;
    ix.code_stride = ((ix.pq_m + 1) / 2 + 15) / 16 * 16;
    ix.row_stride = ix.code_stride;
    dev_alloc(&ix.vectors, (size_t)rows * ix.code_stride);
    dev_alloc((void**)&ix.pq_cb, sizeof(float) * (size_t)ix.pq_m * 16 * 2);
    SOAR_CUDA(cudaMemcpyAsync(ix.pq_cb, pq_cb, sizeof(float) * (size_t)ix.pq_m * 16 * 2, cudaMemcpyDeviceToDevice,
                              s));
    const int ostride = (int)(((d * esz + 15) / 16) * 16 / esz);
    dev_alloc(&ix.originals, esz * (size_t)n * ostride);
    if (dt == SOAR_F32)
      gather_rows<float><<<(unsigned)n, 128, 0, s>>>(static_cast<const float*>(X), d, nullptr, n, ostride,
                                                     static_cast<float*>(ix.originals));
    else
      gather_rows<__nv_bfloat16><<<(unsigned)n, 128, 0, s>>>(static_cast<const __nv_bfloat16*>(X), d, nullptr, n,
                                                             ostride, static_cast<__nv_bfloat16*>(ix.originals));
    SOAR_LAUNCHED();
    pq_encode_index(ix, X, dt, s, scr);
  } else {
    fail(SOAR_EINVAL, "soar_index_build: unknown score mode");
  }

  // one synchronisation: validity flag and the largest partition
  int hbad = 0;
  std::vector<int64_t> off(c + 1);
  SOAR_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  SOAR_CUDA(cudaMemcpyAsync(off.data(), ix.offsets, sizeof(int64_t) * (c + 1), cudaMemcpyDeviceToHost, s));
  SOAR_CUDA(cudaStreamSynchronize(s));
  if (hbad & 1) fail(SOAR_EINVAL, "soar_index_build: an assignment lies outside [0, c)");
  if (hbad & 2) fail(SOAR_EINVAL, "soar_index_build: a point is assigned twice to one partition");
  int64_t mx = 0;
  for (int p = 0; p < c; ++p) mx = std::max(mx, off[p + 1] - off[p]);
  ix.max_partition = mx;

  // partitions ordered by size, largest first (ties by id): the search hands
  // out the longest work items first
  dev_alloc((void**)&ix.part_order, sizeof(int32_t) * c);
  uint32_t* sk = scr.get<uint32_t>(c);
  uint32_t* sk2 = scr.get<uint32_t>(c);
  int32_t* sv2 = scr.get<int32_t>(c);
  size_keys<<<ceil_div(c, 256), 256, 0, s>>>(ix.offsets, c, mx, sk, ix.part_order);
  SOAR_LAUNCHED();
  if (radix_sort_pairs(sk, ix.part_order, sk2, sv2, c, bits_for(mx + 1), s, scr))
    SOAR_CUDA(cudaMemcpyAsync(ix.part_order, sv2, sizeof(int32_t) * c, cudaMemcpyDeviceToDevice, s));

  // full-vector indices also get the tensor-core layout of the rows (fp32
  // rows for the tf32 scan, bf16 rows for the bf16 scan; K padded to one
  // 32-byte MMA step)
  if (ix.mode == SOAR_SCORE_F32) {
    const int kstep = dt == SOAR_F32 ? 8 : 16;
    ix.tc_kp = (d + kstep - 1) / kstep * kstep;
    dev_alloc((void**)&ix.tc_gstart, sizeof(int64_t) * (c + 1));
    group_counts<<<ceil_div((int64_t)c + 1, 256), 256, 0, s>>>(ix.offsets, c, ix.tc_gstart);
    SOAR_LAUNCHED();
    exclusive_scan_i64(ix.tc_gstart, ix.tc_gstart, (int64_t)c + 1, s, scr);
    int64_t groups = 0;
    SOAR_CUDA(cudaMemcpyAsync(&groups, ix.tc_gstart + c, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SOAR_CUDA(cudaStreamSynchronize(s));
    ix.tc_groups = groups;
    dev_alloc(&ix.tc_rows, esz * (size_t)groups * 8 * ix.tc_kp);
    dev_alloc((void**)&ix.tc_ids, sizeof(int32_t) * (size_t)groups * 8);
    dev_alloc((void**)&ix.tc_norms, sizeof(float) * (size_t)groups * 8);
    if (dt == SOAR_F32) {
      fill_tc_rows<float><<<c, 256, 0, s>>>(static_cast<const float*>(ix.vectors), ix.row_stride, d, ix.offsets,
                                            ix.ids, ix.tc_gstart, ix.tc_kp, static_cast<float*>(ix.tc_rows),
                                            ix.tc_ids);
      SOAR_LAUNCHED();
      tc_row_norms<float><<<ceil_div(groups * 8 * 32, 256), 256, 0, s>>>(static_cast<const float*>(ix.tc_rows),
                                                                         groups * 8, ix.tc_kp, ix.tc_norms);
    } else {
      fill_tc_rows<__nv_bfloat16><<<c, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(ix.vectors), ix.row_stride, d,
                                                    ix.offsets, ix.ids, ix.tc_gstart, ix.tc_kp,
                                                    static_cast<__nv_bfloat16*>(ix.tc_rows), ix.tc_ids);
      SOAR_LAUNCHED();
      tc_row_norms<__nv_bfloat16><<<ceil_div(groups * 8 * 32, 256), 256, 0, s>>>(
          static_cast<const __nv_bfloat16*>(ix.tc_rows), groups * 8, ix.tc_kp, ix.tc_norms);
    }
    SOAR_LAUNCHED();
    dev_alloc((void**)&ix.tc_pmax, sizeof(float) * c);
    partition_max_norm<<<c, 256, 0, s>>>(ix.tc_norms, ix.tc_gstart, ix.tc_pmax);
    SOAR_LAUNCHED();
  }
  // fp32 centroid scores: the codebook packed for the tensor-core selection
  if (ix.mode != SOAR_SCORE_FP8 && select_tc_fits((d + 7) / 8 * 8)) {
    ix.sel_kp = (d + 7) / 8 * 8;
    ix.sel_tiles = (c + 63) / 64;
    dev_alloc((void**)&ix.sel_cb, sizeof(float) * 2 * 64 * (size_t)ix.sel_kp * ix.sel_tiles);
    pack_select_codebook(ix, ix.sel_cb, s);
  }
  SOAR_CUDA(cudaStreamSynchronize(s));
}

void free_index(IndexData& ix) {
  void* ptrs[] = {ix.offsets, ix.ids, ix.vectors, ix.row_scales, ix.originals, ix.centroids,
                  ix.part_order, ix.cent_code_vals, ix.cent_scales, ix.tc_rows, ix.tc_gstart,
                  ix.tc_ids, ix.tc_norms, ix.tc_pmax, ix.assign, ix.sel_cb, ix.pq_cb};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  ix = IndexData{};
}

}  // namespace soar
