// C ABI of the library (declared in include/soar.h): argument checks,
// error translation and the index handle.  All compute lives in the other
// translation units; nothing here touches vector data on the host.
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "scan_common.cuh"

namespace soar {

std::atomic<uint64_t> g_launches{0};

namespace {
struct StageEvent {
  std::string stage;
  cudaEvent_t begin, end;
};
std::mutex g_stage_mu;
bool g_stage_on = false;
std::vector<StageEvent> g_stage_events;
std::vector<std::pair<std::string, cudaEvent_t>> g_open;
}  // namespace

void stage_mark(cudaStream_t s, const char* stage, bool begin) {
  std::lock_guard<std::mutex> lock(g_stage_mu);
  if (!g_stage_on) return;
  cudaEvent_t e;
  SOAR_CUDA(cudaEventCreate(&e));
  SOAR_CUDA(cudaEventRecord(e, s));
  if (begin) {
    g_open.emplace_back(stage, e);
    return;
  }
  for (size_t i = g_open.size(); i-- > 0;) {
    if (g_open[i].first == stage) {
      g_stage_events.push_back(StageEvent{stage, g_open[i].second, e});
      g_open.erase(g_open.begin() + (long)i);
      return;
    }
  }
  cudaEventDestroy(e);
}

namespace {
// The device error word: a static device variable (zero at module load), so
// that no call, the allocation-free ones included, allocates it.  Its device
// address is looked up once per device with cudaGetSymbolAddress.
__device__ int g_err_dev;
std::mutex g_err_mu;
int* g_err_word[256] = {};
}  // namespace

int* device_error_word() {
  int dev = 0;
  SOAR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) fail(SOAR_EUNSUPPORTED, "device ordinal above 255");
  std::lock_guard<std::mutex> lock(g_err_mu);
  if (!g_err_word[dev]) {
    void* p = nullptr;
    SOAR_CUDA(cudaGetSymbolAddress(&p, g_err_dev));
    g_err_word[dev] = static_cast<int*>(p);
  }
  return g_err_word[dev];
}

}  // namespace soar

namespace {

thread_local std::string g_last_error;

// Keep freed pool memory cached so per-call scratch costs no driver calls.
void configure_pool() {
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    uint64_t threshold = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
  });
}

template <typename F>
soar_status guarded(F&& f) {
  try {
    configure_pool();
    f();
    g_last_error.clear();
    return SOAR_OK;
  } catch (const soar::Error& e) {
    g_last_error = e.what();
    return e.status;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return SOAR_ENOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return SOAR_ECUDA;
  } catch (...) {
    g_last_error = "unknown error";
    return SOAR_ECUDA;
  }
}

bool valid_dtype(soar_dtype dt) { return dt == SOAR_F32 || dt == SOAR_BF16; }

// Scratch of soar_select_partitions_static: a fixed device array that every
// GPU loading this library holds until the process exits.  Host code must not
// use `g_static_scratch` as an address (on the host it names a stand-in); the
// device address is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[SOAR_STATIC_SCRATCH_BYTES];

std::mutex g_static_mu;
void* g_static_ptr[256] = {};

// Device address of g_static_scratch on the current device (looked up on the
// first call made with that device current).
void* static_scratch() {
  int dev = 0;
  SOAR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) soar::fail(SOAR_EUNSUPPORTED, "device ordinal above 255");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    SOAR_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_ptr[dev] = p;
  }
  return g_static_ptr[dev];
}

// A coarse index usable over an index of c fine partitions in d dimensions:
// its rows are that index's fine centroids.
void require_coarse_of(const soar_index* coarse, int32_t c, int32_t d) {
  const soar::IndexData& x = coarse->data;
  SOAR_REQUIRE(x.n == c && x.d == d, "the coarse index's rows must be the c fine centroids (n == c, same d)");
  SOAR_REQUIRE(x.mode == SOAR_SCORE_F32 && x.dtype == SOAR_F32, "the coarse index must hold fp32 rows");
}

}  // namespace

extern "C" {

const char* soar_last_error(void) { return g_last_error.c_str(); }

const char* soar_version(void) { return "soar-gb300 0.1 sm_103a"; }

soar_status soar_train_centroids(const void* X, soar_dtype dtype, int64_t n, int32_t d, int32_t c, int32_t iters,
                                 const int32_t* init_idx, float* C_out, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(X && init_idx && C_out, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    SOAR_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "n must be in [1, 2^31)");
    SOAR_REQUIRE(d >= 1 && d <= 4096, "d must be in [1, 4096]");
    SOAR_REQUIRE(c >= 1 && c <= n, "c must be in [1, n]");
    SOAR_REQUIRE(iters >= 0, "iters must be >= 0");
    soar::Scratch scr(stream);
    soar::kmeans_train(X, dtype, n, d, c, iters, init_idx, C_out, stream, scr);
  });
}

soar_status soar_assign(const void* X, soar_dtype dtype, int64_t n, int32_t d, const float* C, int32_t c,
                        float lambda, int32_t spills, int32_t* assign_out, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(X && C && assign_out, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    SOAR_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "n must be in [1, 2^31)");
    SOAR_REQUIRE(d >= 1 && d <= 4096, "d must be in [1, 4096]");
    SOAR_REQUIRE(std::isfinite(lambda) && lambda >= 0.f, "lambda must be finite and >= 0");
    SOAR_REQUIRE(spills >= 0 && spills <= 4, "spills must be in [0, 4]");
    SOAR_REQUIRE(c >= 1 + spills, "c must be >= 1 + spills");
    soar::Scratch scr(stream);
    soar::assign_points(X, dtype, n, d, C, c, lambda, spills, assign_out, stream, scr);
  });
}

soar_status soar_index_build(const void* X, soar_dtype dtype, int64_t n, int32_t d, const float* C, int32_t c,
                             const int32_t* assign, int32_t spills, soar_score_mode mode, soar_index** out,
                             cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(X && C && assign && out, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    SOAR_REQUIRE(n >= 1 && d >= 1 && d <= 4096 && c >= 1, "bad sizes");
    SOAR_REQUIRE(spills >= 0 && spills <= 4 && c >= 1 + spills, "spills must be in [0, 4] and <= c - 1");
    SOAR_REQUIRE(n * (1 + spills) < (int64_t(1) << 31), "n * (1 + spills) must be < 2^31");
    SOAR_REQUIRE(mode == SOAR_SCORE_F32 || mode == SOAR_SCORE_FP8 || mode == SOAR_SCORE_PQ4, "unknown mode");
    SOAR_REQUIRE(mode != SOAR_SCORE_PQ4, "a SOAR_SCORE_PQ4 index needs its codebooks: use soar_index_build_pq");
    soar_index* ix = new soar_index;
    ix->data.n = n;
    ix->data.d = d;
    ix->data.c = c;
    ix->data.spills = spills;
    ix->data.mode = mode;
    ix->data.dtype = dtype;
    ix->data.rows = n * (1 + spills);
    try {
      soar::build_index(ix->data, X, dtype, C, assign, stream);
    } catch (...) {
      cudaStreamSynchronize(stream);
      soar::free_index(ix->data);
      delete ix;
      throw;
    }
    *out = ix;
  });
}

soar_status soar_pq_train(const void* X, soar_dtype dtype, int64_t n, int32_t d, const float* C, int32_t c,
                          const int32_t* part, int32_t iters, const int32_t* init_idx, float* B_out,
                          cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(X && C && part && init_idx && B_out, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    SOAR_REQUIRE(n >= 16 && n < (int64_t(1) << 31), "n must be in [16, 2^31)");
    SOAR_REQUIRE(d >= 2 && d <= 4096 && d % 2 == 0, "d must be even and in [2, 4096]");
    SOAR_REQUIRE(c >= 1, "c must be >= 1");
    SOAR_REQUIRE(iters >= 0, "iters must be >= 0");
    SOAR_REQUIRE(n * (int64_t)d < (int64_t(1) << 40), "n * d too large");
    soar::Scratch scr(stream);
    soar::pq_train(X, dtype, n, d, C, part, iters, init_idx, B_out, stream, scr);
  });
}

soar_status soar_index_build_pq(const void* X, soar_dtype dtype, int64_t n, int32_t d, const float* C, int32_t c,
                                const int32_t* assign, int32_t spills, const float* B, soar_index** out,
                                cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(X && C && assign && B && out, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    SOAR_REQUIRE(n >= 1 && d >= 2 && d <= 4096 && d % 2 == 0 && c >= 1, "bad sizes (d must be even)");
    SOAR_REQUIRE(spills >= 0 && spills <= 4 && c >= 1 + spills, "spills must be in [0, 4] and <= c - 1");
    SOAR_REQUIRE(n * (1 + spills) < (int64_t(1) << 31), "n * (1 + spills) must be < 2^31");
    soar_index* ix = new soar_index;
    ix->data.n = n;
    ix->data.d = d;
    ix->data.c = c;
    ix->data.spills = spills;
    ix->data.mode = SOAR_SCORE_PQ4;
    ix->data.dtype = dtype;
    ix->data.rows = n * (1 + spills);
    try {
      soar::build_index(ix->data, X, dtype, C, assign, stream, B);
    } catch (...) {
      cudaStreamSynchronize(stream);
      soar::free_index(ix->data);
      delete ix;
      throw;
    }
    *out = ix;
  });
}

soar_status soar_index_get_info(const soar_index* index, soar_index_info* info) {
  return guarded([&] {
    SOAR_REQUIRE(index && info, "null pointer");
    const soar::IndexData& x = index->data;
    info->n = x.n;
    info->d = x.d;
    info->c = x.c;
    info->spills = x.spills;
    info->mode = x.mode;
    info->dtype = x.dtype;
    info->row_stride = x.row_stride;
    info->rows = x.rows;
    info->max_partition = x.max_partition;
    info->offsets = x.offsets;
    info->ids = x.ids;
    info->vectors = x.vectors;
    info->row_scales = x.row_scales;
    info->originals = x.originals;
    info->centroids = x.centroids;
    info->device_bytes = x.bytes;
  });
}

soar_status soar_index_free(soar_index* index) {
  return guarded([&] {
    if (!index) return;
    SOAR_CUDA(cudaDeviceSynchronize());
    soar::free_index(index->data);
    delete index;
  });
}

soar_status soar_index_save(const soar_index* index, const char* path, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(index && path, "null pointer");
    soar::save_index(index->data, path, stream);
  });
}

soar_status soar_index_load(const char* path, soar_index** out, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(path && out, "null pointer");
    soar_index* ix = new soar_index;
    try {
      soar::load_index(ix->data, path, stream);
    } catch (...) {
      cudaStreamSynchronize(stream);
      soar::free_index(ix->data);
      delete ix;
      throw;
    }
    *out = ix;
  });
}

soar_status soar_select_partitions(const soar_index* index, const void* Q, soar_dtype dtype, int64_t nq, int32_t t,
                                   int32_t* top_out, float* score_out, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(index && Q && top_out, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    SOAR_REQUIRE(nq >= 1 && nq < (int64_t(1) << 31), "nq must be in [1, 2^31)");
    SOAR_REQUIRE(t >= 1 && t <= index->data.c && t <= 8192, "t must be in [1, min(c, 8192)]");
    soar::Scratch scr(stream);
    soar::select_partitions(index->data, Q, dtype, nq, t, top_out, score_out, stream, scr);
  });
}

soar_status soar_search(const soar_index* index, const void* Q, soar_dtype dtype, int64_t nq, int32_t k, int32_t t,
                        const int32_t* t_per_query, int32_t rescore, int64_t* ids_out, float* scores_out,
                        cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(index && Q && ids_out && scores_out, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    SOAR_REQUIRE(nq >= 1 && nq * (int64_t)t < (int64_t(1) << 31), "nq * t must be in [1, 2^31)");
    SOAR_REQUIRE(k >= 1 && k <= 1024, "k must be in [1, 1024]");
    SOAR_REQUIRE(t >= 1 && t <= index->data.c && t <= 8192, "t must be in [1, min(c, 8192)]");
    if (index->data.mode == SOAR_SCORE_FP8 || index->data.mode == SOAR_SCORE_PQ4)
      SOAR_REQUIRE(rescore >= k && rescore <= 4096, "rescore must be in [k, 4096] for an FP8 or PQ4 index");
    soar::Scratch scr(stream);
    soar::search(index->data, Q, dtype, nq, k, t, t_per_query, rescore, ids_out, scores_out, stream, scr);
  });
}

soar_status soar_index_build_coarse(const soar_index* index, int32_t c2, int32_t iters, const int32_t* init_idx,
                                   float lambda, int32_t spills, soar_index** out, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(index && init_idx && out, "null pointer");
    const soar::IndexData& fine = index->data;
    SOAR_REQUIRE(c2 >= 1 + spills && c2 <= fine.c, "c2 must be in [1 + spills, c]");
    SOAR_REQUIRE(iters >= 0, "iters must be >= 0");
    SOAR_REQUIRE(std::isfinite(lambda) && lambda >= 0.f, "lambda must be finite and >= 0");
    SOAR_REQUIRE(spills >= 0 && spills <= 4, "spills must be in [0, 4]");
    soar::Scratch scr(stream);
    float* C2 = scr.get<float>((size_t)c2 * fine.d);
    int32_t* A2 = scr.get<int32_t>((size_t)fine.c * (1 + spills));
    soar::kmeans_train(fine.centroids, SOAR_F32, fine.c, fine.d, c2, iters, init_idx, C2, stream, scr);
    soar::assign_points(fine.centroids, SOAR_F32, fine.c, fine.d, C2, c2, lambda, spills, A2, stream, scr);
    soar_index* ix = new soar_index;
    ix->data.n = fine.c;
    ix->data.d = fine.d;
    ix->data.c = c2;
    ix->data.spills = spills;
    ix->data.mode = SOAR_SCORE_F32;
    ix->data.dtype = SOAR_F32;
    ix->data.rows = (int64_t)fine.c * (1 + spills);
    try {
      soar::build_index(ix->data, fine.centroids, SOAR_F32, C2, A2, stream);
    } catch (...) {
      cudaStreamSynchronize(stream);
      soar::free_index(ix->data);
      delete ix;
      throw;
    }
    *out = ix;
  });
}

soar_status soar_select_partitions_multilevel(const soar_index* coarse, const void* Q, soar_dtype dtype, int64_t nq,
                                              int32_t t, int32_t t1, int32_t* top_out, float* score_out,
                                              int32_t* count_out, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(coarse && Q && top_out && count_out, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    const soar::IndexData& x = coarse->data;
    SOAR_REQUIRE(x.mode == SOAR_SCORE_F32 && x.dtype == SOAR_F32, "the coarse index must hold fp32 rows");
    SOAR_REQUIRE(nq >= 1 && nq * (int64_t)t < (int64_t(1) << 31) && nq * (int64_t)t1 < (int64_t(1) << 31),
                 "nq * t and nq * t1 must be < 2^31");
    SOAR_REQUIRE(t >= 1 && t <= x.n && t <= 1024, "t must be in [1, min(c, 1024)]");
    SOAR_REQUIRE(t1 >= 1 && t1 <= x.c && t1 <= 8192, "t1 must be in [1, min(c2, 8192)]");
    soar::Scratch scr(stream);
    soar::multilevel_select(x, Q, dtype, nq, t, t1, top_out, score_out, count_out, stream, scr);
  });
}

soar_status soar_search_multilevel(const soar_index* index, const soar_index* coarse, const void* Q,
                                   soar_dtype dtype, int64_t nq, int32_t k, int32_t t, int32_t t1, int32_t rescore,
                                   int64_t* ids_out, float* scores_out, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(index && coarse && Q && ids_out && scores_out, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    require_coarse_of(coarse, index->data.c, index->data.d);
    SOAR_REQUIRE(nq >= 1 && nq * (int64_t)t < (int64_t(1) << 31) && nq * (int64_t)t1 < (int64_t(1) << 31),
                 "nq * t and nq * t1 must be < 2^31");
    SOAR_REQUIRE(k >= 1 && k <= 1024, "k must be in [1, 1024]");
    SOAR_REQUIRE(t >= 1 && t <= index->data.c && t <= 1024, "t must be in [1, min(c, 1024)]");
    SOAR_REQUIRE(t1 >= 1 && t1 <= coarse->data.c && t1 <= 8192, "t1 must be in [1, min(c2, 8192)]");
    if (index->data.mode == SOAR_SCORE_FP8 || index->data.mode == SOAR_SCORE_PQ4)
      SOAR_REQUIRE(rescore >= k && rescore <= 4096, "rescore must be in [k, 4096] for an FP8 or PQ4 index");
    soar::Scratch scr(stream);
    soar::search(index->data, Q, dtype, nq, k, t, nullptr, rescore, ids_out, scores_out, stream, scr, &coarse->data,
                 t1);
  });
}

soar_status soar_merge_topk(const int64_t* ids, const float* scores, int64_t nq, int32_t m, int32_t len,
                            const int64_t* id_offsets, int32_t k, int64_t* ids_out, float* scores_out,
                            cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(ids && scores && ids_out && scores_out, "null pointer");
    SOAR_REQUIRE(nq >= 1 && m >= 1 && m <= 4096 && len >= 1 && len <= 1024 && k >= 1 && k <= 1024, "bad sizes");
    SOAR_REQUIRE(nq * (int64_t)m * len < (int64_t(1) << 40), "too many list entries");
    soar::Scratch scr(stream);
    soar::merge_topk(ids, scores, nq, m, len, id_offsets, k, ids_out, scores_out, stream, scr);
  });
}

soar_status soar_exact_mips(const void* X, soar_dtype xdtype, int64_t n, int32_t d, const void* Q, soar_dtype qdtype,
                            int64_t nq, int32_t k, int64_t* ids_out, float* scores_out, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(X && Q && ids_out && scores_out, "null pointer");
    SOAR_REQUIRE(valid_dtype(xdtype) && valid_dtype(qdtype), "unknown dtype");
    SOAR_REQUIRE(n >= 1 && n < (int64_t(1) << 31) && nq >= 1 && d >= 1 && d <= 4096, "bad sizes");
    SOAR_REQUIRE(k >= 1 && k <= 1024, "k must be in [1, 1024]");
    soar::Scratch scr(stream);
    soar::exact_mips(X, xdtype, n, d, Q, qdtype, nq, k, ids_out, scores_out, stream, scr);
  });
}

soar_status soar_select_partitions_static(const soar_index* index, const void* Q, soar_dtype dtype, int64_t nq,
                                          int32_t t, int32_t* top_out, float* score_out, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(index && Q && top_out, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    SOAR_REQUIRE(nq >= 1 && nq < (int64_t(1) << 31), "nq must be in [1, 2^31)");
    SOAR_REQUIRE(t >= 1 && t <= index->data.c && t <= 8192, "t must be in [1, min(c, 8192)]");
    const size_t need = soar::select_scratch_bytes(index->data, nq);
    if (need > (size_t)SOAR_STATIC_SCRATCH_BYTES)
      soar::fail(SOAR_EINVAL, "soar_select_partitions_static: " + std::to_string(nq) + " queries need " +
                                  std::to_string(need) + " bytes of scratch, more than the " +
                                  std::to_string((size_t)SOAR_STATIC_SCRATCH_BYTES) +
                                  "-byte static buffer; pass fewer queries per call");
    soar::select_partitions_in(index->data, Q, dtype, nq, t, top_out, score_out, static_scratch(), stream);
  });
}

int64_t soar_mlp_param_count(int32_t d_in, int32_t hidden) {
  return d_in > 0 && hidden > 0 ? soar::mlp_param_count(d_in, hidden) : -1;
}

soar_status soar_probe_features(const soar_index* index, const void* Q, soar_dtype dtype, int64_t nq, int32_t top,
                                float* Z_out, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(index && Q && Z_out, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    SOAR_REQUIRE(nq >= 1 && top >= 1 && top <= index->data.c && top <= 8192, "bad sizes");
    soar::Scratch scr(stream);
    soar::probe_features(index->data, Q, dtype, nq, top, Z_out, stream, scr);
  });
}

soar_status soar_probe_labels(const soar_index* index, const void* Q, soar_dtype dtype, int64_t nq,
                              const int64_t* truth_ids, int32_t k, float target_recall, int32_t* labels_out,
                              cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(index && Q && truth_ids && labels_out, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    SOAR_REQUIRE(nq >= 1 && k >= 1 && k <= 1024, "bad sizes");
    SOAR_REQUIRE(target_recall > 0.f && target_recall <= 1.f, "target_recall must be in (0, 1]");
    soar::Scratch scr(stream);
    soar::probe_labels(index->data, Q, dtype, nq, truth_ids, k, target_recall, labels_out, stream, scr);
  });
}

soar_status soar_mlp_forward(const float* params, int32_t d_in, int32_t hidden, const float* Z, int32_t batch,
                             int32_t bf16, float* y_out, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(params && Z && y_out, "null pointer");
    SOAR_REQUIRE(d_in >= 1 && hidden >= 1 && batch >= 1, "bad sizes");
    soar::Scratch scr(stream);
    soar::mlp_predict(params, d_in, hidden, Z, batch, bf16 != 0, 1.f, 1, y_out, nullptr, stream, scr);
  });
}

soar_status soar_mlp_backward(const float* params, int32_t d_in, int32_t hidden, const float* Z, const float* target,
                              int32_t batch, int32_t bf16, float* grads_out, float* loss_out, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(params && Z && target && grads_out, "null pointer");
    SOAR_REQUIRE(d_in >= 1 && hidden >= 1 && batch >= 1, "bad sizes");
    soar::Scratch scr(stream);
    soar::mlp_backward(params, d_in, hidden, Z, target, batch, bf16 != 0, grads_out, loss_out, stream, scr);
  });
}

soar_status soar_mlp_adam(float* params, const float* grads, float* m1, float* m2, int64_t count, int32_t step,
                          float lr, float beta1, float beta2, float eps, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(params && grads && m1 && m2, "null pointer");
    SOAR_REQUIRE(count >= 1 && step >= 1 && std::isfinite(lr), "bad arguments");
    soar::mlp_adam(params, grads, m1, m2, count, step, lr, beta1, beta2, eps, stream);
  });
}

soar_status soar_mlp_predict_probes(const float* params, int32_t d_in, int32_t hidden, const float* Z, int32_t batch,
                                    int32_t bf16, float alpha, int32_t c, int32_t* t_out, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(params && Z && t_out, "null pointer");
    SOAR_REQUIRE(d_in >= 1 && hidden >= 1 && batch >= 1 && c >= 1, "bad sizes");
    SOAR_REQUIRE(std::isfinite(alpha) && alpha > 0.f, "alpha must be finite and > 0");
    soar::Scratch scr(stream);
    soar::mlp_predict(params, d_in, hidden, Z, batch, bf16 != 0, alpha, c, nullptr, t_out, stream, scr);
  });
}

soar_status soar_search_learned(const soar_index* index, const void* Q, soar_dtype dtype, int64_t nq, int32_t k,
                                int32_t top, const float* params, int32_t hidden, int32_t bf16, float alpha,
                                int32_t t_cap, int32_t rescore, int64_t* ids_out, float* scores_out, int32_t* t_out,
                                cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(index && Q && params && ids_out && scores_out, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    SOAR_REQUIRE(nq >= 1 && nq * (int64_t)top < (int64_t(1) << 31) && nq < (int64_t(1) << 31),
                 "nq * top must be in [1, 2^31)");
    SOAR_REQUIRE(k >= 1 && k <= 1024, "k must be in [1, 1024]");
    SOAR_REQUIRE(top >= 1 && top <= index->data.c && top <= 8192, "top must be in [1, min(c, 8192)]");
    SOAR_REQUIRE(t_cap >= 1 && t_cap <= top, "t_cap must be in [1, top]");
    SOAR_REQUIRE(hidden >= 1, "hidden must be >= 1");
    SOAR_REQUIRE(std::isfinite(alpha) && alpha > 0.f, "alpha must be finite and > 0");
    if (index->data.mode == SOAR_SCORE_FP8 || index->data.mode == SOAR_SCORE_PQ4)
      SOAR_REQUIRE(rescore >= k && rescore <= 4096, "rescore must be in [k, 4096] for an FP8 or PQ4 index");
    soar::Scratch scr(stream);
    const soar::LearnedProbe lp{params, index->data.d + top, hidden, bf16 != 0, alpha, t_cap, t_out};
    soar::search(index->data, Q, dtype, nq, k, top, nullptr, rescore, ids_out, scores_out, stream, scr, nullptr, 0,
                 &lp);
  });
}

soar_status soar_check_device(void) {
  return guarded([&] {
    SOAR_CUDA(cudaDeviceSynchronize());
    int* w = soar::device_error_word();
    int v = 0;
    SOAR_CUDA(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost));
    if (v) {
      SOAR_CUDA(cudaMemset(w, 0, sizeof(int)));
      soar::fail(SOAR_ETIMEOUT, "a kernel gave up a bounded wait (device work of an earlier call is incomplete)");
    }
  });
}

uint64_t soar_kernel_launches(void) { return soar::g_launches.load(); }

soar_status soar_set_wait_limit(int64_t cycles) {
  return guarded([&] {
    SOAR_REQUIRE(cycles >= 0, "cycles must be >= 0");
    soar::set_scan_wait_limit(cycles);
  });
}

soar_status soar_stage_timing(int enable) {
  return guarded([&] {
    std::lock_guard<std::mutex> lock(soar::g_stage_mu);
    soar::g_stage_on = enable != 0;
  });
}

int soar_stage_times(char* names, int names_len, float* ms, int* launches, int max_stages) {
  std::lock_guard<std::mutex> lock(soar::g_stage_mu);
  std::vector<std::string> order;
  std::vector<float> tot;
  std::vector<int> cnt;
  for (auto& ev : soar::g_stage_events) {
    float t = 0.f;
    if (cudaEventSynchronize(ev.end) == cudaSuccess) cudaEventElapsedTime(&t, ev.begin, ev.end);
    cudaEventDestroy(ev.begin);
    cudaEventDestroy(ev.end);
    size_t i = 0;
    while (i < order.size() && order[i] != ev.stage) ++i;
    if (i == order.size()) {
      order.push_back(ev.stage);
      tot.push_back(0.f);
      cnt.push_back(0);
    }
    tot[i] += t;
    cnt[i] += 1;
  }
  soar::g_stage_events.clear();
  std::string joined;
  int m = 0;
  for (size_t i = 0; i < order.size() && m < max_stages; ++i, ++m) {
    if (ms) ms[m] = tot[i];
    if (launches) launches[m] = cnt[i];
    joined += (i ? "," : "") + order[i];
  }
  if (names && names_len > 0) {
    size_t n = std::min((size_t)names_len - 1, joined.size());
    memcpy(names, joined.data(), n);
    names[n] = 0;
  }
  return m;
}

soar_status soar_quantize_fp8(const void* V, soar_dtype dtype, int64_t m, int32_t d, uint8_t* codes,
                              int32_t code_stride, float* scales, cudaStream_t stream) {
  return guarded([&] {
    SOAR_REQUIRE(V && codes && scales, "null pointer");
    SOAR_REQUIRE(valid_dtype(dtype), "unknown dtype");
    SOAR_REQUIRE(m >= 0 && d >= 1 && code_stride >= d, "bad sizes");
    soar::quantize_fp8(V, dtype, m, d, codes, code_stride, scales, stream);
  });
}

}  // extern "C"
