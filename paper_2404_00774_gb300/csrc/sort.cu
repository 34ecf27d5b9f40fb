// Device-wide prefix sums and a stable LSD radix sort of (small key, value)
// pairs.  The sort keeps equal keys in input order, which is what makes the
// inverted lists list their members in ascending point id and groups search
// work by partition deterministically.
#include "internal.cuh"

namespace soar {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_tile_sums(const T* in, T* sums, int64_t count) {
  __shared__ T warp[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < count) s += in[base + i];
  T total;
  block_exclusive_scan<T>(s, warp, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Single block: exclusive scan of the tile sums in place, carrying across chunks.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_sums_inplace(T* sums, int64_t nb) {
  __shared__ T warp[32];
  T carry = 0;
  for (int64_t c0 = 0; c0 < nb; c0 += kScanThreads) {
    int64_t i = c0 + threadIdx.x;
    T v = i < nb ? sums[i] : T(0);
    T total;
    T ex = block_exclusive_scan<T>(v, warp, total);
    if (i < nb) sums[i] = carry + ex;
    carry += total;
  }
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_apply(const T* in, T* out, const T* sums,
                                                           int64_t count) {
  __shared__ T warp[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < count ? in[base + i] : T(0);
    s += v[i];
  }
  T total;
  T run = block_exclusive_scan<T>(s, warp, total) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < count) out[base + i] = run;
    run += v[i];
  }
}

template <typename T>
void exclusive_scan(const T* in, T* out, int64_t count, cudaStream_t s, Scratch& scr) {
  if (count <= 0) return;
  int64_t nb = (count + kScanTile - 1) / kScanTile;
  T* sums = scr.get<T>(nb);
  scan_tile_sums<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, sums, count);
  SOAR_LAUNCHED();
  scan_sums_inplace<T><<<1, kScanThreads, 0, s>>>(sums, nb);
  SOAR_LAUNCHED();
  scan_apply<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, sums, count);
  SOAR_LAUNCHED();
}

// ------------------------------------------------------------- radix sort

constexpr int kRsThreads = 256;
constexpr int kRsRounds = 8;
constexpr int kRsTile = kRsThreads * kRsRounds;   // elements per block; element e of a
                                                  // tile sits at round e/256, thread e%256

__global__ void __launch_bounds__(kRsThreads) rs_hist(const uint32_t* keys, int64_t count, int shift,
                                                      int32_t* hist, int nblocks) {
  __shared__ int32_t h[256];
  const int tid = threadIdx.x;
  h[tid] = 0;
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * kRsTile;
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    int64_t e = tile0 + r * kRsThreads + tid;
    if (e < count) atomicAdd(&h[(keys[e] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(int64_t)tid * nblocks + blockIdx.x] = h[tid];   // digit-major
}

// Stable scatter: the rank of an element among equal digits of its tile is
// (earlier rounds) + (earlier warps of this round) + (earlier lanes of its warp).
__global__ void __launch_bounds__(kRsThreads) rs_scatter(const uint32_t* keys, const int32_t* vals,
                                                         int64_t count, int shift, const int32_t* base,
                                                         int nblocks, uint32_t* keys_out,
                                                         int32_t* vals_out) {
  constexpr int W = kRsThreads / 32;
  __shared__ int32_t warp_cnt[W][256];
  __shared__ int32_t warp_pre[W][256];
  __shared__ int32_t gbase[256];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  gbase[tid] = base[(int64_t)tid * nblocks + blockIdx.x];
  int32_t tile_cnt = 0;  // owned by the thread whose index equals the digit
#pragma unroll
  for (int ww = 0; ww < W; ++ww) warp_cnt[ww][tid] = 0;
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  const int64_t tile0 = (int64_t)blockIdx.x * kRsTile;
  for (int r = 0; r < kRsRounds; ++r) {
    const int64_t e = tile0 + r * kRsThreads + tid;
    const bool valid = e < count;
    const uint32_t key = valid ? keys[e] : 0u;
    const int32_t val = valid ? vals[e] : 0;
    const int dig = valid ? (int)((key >> shift) & 255u) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, dig);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) warp_cnt[w][dig] = __popc(peers);
    __syncthreads();
    int32_t run = tile_cnt;
#pragma unroll
    for (int ww = 0; ww < W; ++ww) {
      int32_t c = warp_cnt[ww][tid];
      warp_pre[ww][tid] = run;
      run += c;
      warp_cnt[ww][tid] = 0;
    }
    tile_cnt = run;
    __syncthreads();
    if (valid) {
      const int32_t pos = gbase[dig] + warp_pre[w][dig] + rank;
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
  }
}

__global__ void seg_offsets_kernel(const uint32_t* keys, int64_t count, int32_t num_keys,
                                   int64_t* offsets) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > num_keys) return;
  int64_t lo = 0, hi = count;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (keys[mid] < (uint32_t)p) lo = mid + 1; else hi = mid;
  }
  offsets[p] = lo;
}

}  // namespace

void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t count, cudaStream_t s, Scratch& scr) {
  exclusive_scan<int32_t>(in, out, count, s, scr);
}
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t count, cudaStream_t s, Scratch& scr) {
  exclusive_scan<int64_t>(in, out, count, s, scr);
}

int bits_for(int64_t num_keys) {
  int b = 1;
  while (b < 40 && ((int64_t)1 << b) < num_keys) ++b;
  return b;
}

bool radix_sort_pairs(uint32_t* keys, int32_t* vals, uint32_t* keys_tmp, int32_t* vals_tmp,
                      int64_t count, int key_bits, cudaStream_t s, Scratch& scr) {
  if (count <= 0) return false;
  if (count >= ((int64_t)1 << 31)) fail(SOAR_EUNSUPPORTED, "radix_sort_pairs: more than 2^31 - 1 pairs");
  const int nblocks = (int)((count + kRsTile - 1) / kRsTile);
  int32_t* hist = scr.get<int32_t>((size_t)256 * nblocks);
  bool in_tmp = false;
  for (int shift = 0; shift < key_bits; shift += 8) {
    uint32_t* ki = in_tmp ? keys_tmp : keys;
    int32_t* vi = in_tmp ? vals_tmp : vals;
    uint32_t* ko = in_tmp ? keys : keys_tmp;
    int32_t* vo = in_tmp ? vals : vals_tmp;
    rs_hist<<<nblocks, kRsThreads, 0, s>>>(ki, count, shift, hist, nblocks);
    SOAR_LAUNCHED();
    exclusive_scan<int32_t>(hist, hist, (int64_t)256 * nblocks, s, scr);
    rs_scatter<<<nblocks, kRsThreads, 0, s>>>(ki, vi, count, shift, hist, nblocks, ko, vo);
    SOAR_LAUNCHED();
    in_tmp = !in_tmp;
  }
  return in_tmp;
}

void segment_offsets(const uint32_t* keys_sorted, int64_t count, int32_t num_keys, int64_t* offsets,
                     cudaStream_t s) {
  seg_offsets_kernel<<<ceil_div(num_keys + 1, 256), 256, 0, s>>>(keys_sorted, count, num_keys, offsets);
  SOAR_LAUNCHED();
}

}  // namespace soar
