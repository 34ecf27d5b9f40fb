// Internal launchers shared between the translation units of the library.
#pragma once

#include "common.cuh"

namespace soar {

// A per-device int that kernels set when a bounded wait expired (api.cu);
// soar_check_device() reads and clears it.
int* device_error_word();

// ----------------------------------------------------------- sort.cu

// Exclusive prefix sum of `count` values; out may alias in.  Returns nothing;
// the total is out[count-1] + in[count-1] (callers that need it keep a copy).
void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t count, cudaStream_t s, Scratch& scr);
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t count, cudaStream_t s, Scratch& scr);

// Stable sort of (key, value) pairs by key, keys in [0, 2^key_bits).
// Ping-pongs between (keys, vals) and (keys_tmp, vals_tmp); returns true when
// the sorted result ended in the *_tmp buffers.
bool radix_sort_pairs(uint32_t* keys, int32_t* vals, uint32_t* keys_tmp, int32_t* vals_tmp,
                      int64_t count, int key_bits, cudaStream_t s, Scratch& scr);

// offsets[p] = first position whose key >= p, for p in [0, num_keys]; keys sorted.
void segment_offsets(const uint32_t* keys_sorted, int64_t count, int32_t num_keys,
                     int64_t* offsets, cudaStream_t s);

int bits_for(int64_t num_keys);

// ----------------------------------------------------------- assign.cu

// pi(x) for every row (nearest centroid, lower index on ties), optionally the
// SOAR spills, written to assign[n][1+spills].
void assign_points(const void* X, soar_dtype dt, int64_t n, int32_t d, const float* C, int32_t c,
                   float lambda, int32_t spills, int32_t* assign, cudaStream_t s, Scratch& scr);

void kmeans_train(const void* X, soar_dtype dt, int64_t n, int32_t d, int32_t c, int32_t iters,
                  const int32_t* init_idx, float* C, cudaStream_t s, Scratch& scr);

// Tensor-core assignment pass (assign_tc.cu): the primary assignment
// (ndir = 0) or the first spill (ndir = 1, inv_rn[n][4] column 0 from the
// residual kernel), written to column ndir of assign[n][astride].
bool assign_tc_supported(int d, int ndir);
template <typename XT>
void assign_tc_pass(const XT* X, int64_t n, int d, const float* C, int c, int ndir, int32_t* assign, int astride,
                    const float* inv_rn, float lambda, cudaStream_t s, Scratch& scr);

// ----------------------------------------------------------- ivf.cu

struct IndexData {
  int64_t n = 0;
  int32_t d = 0, c = 0, spills = 0, mode = 0, dtype = 0, row_stride = 0;
  int64_t rows = 0, max_partition = 0, bytes = 0;
  int64_t* offsets = nullptr;   // [c+1]
  int32_t* ids = nullptr;       // [rows]
  void* vectors = nullptr;      // [rows][row_stride]
  float* row_scales = nullptr;  // [rows] (FP8)
  void* originals = nullptr;    // [n][row_stride] (FP8)
  float* centroids = nullptr;   // [c][d]
  int32_t* part_order = nullptr;  // [c] partitions by size, largest first
  float* cent_code_vals = nullptr;  // [c][code_stride] decoded E4M3 code values (FP8)
  float* cent_scales = nullptr;     // [c] (FP8)
  int32_t code_stride = 0;
  // rows for the tensor-core scan in the stored dtype (fp32 or bf16): each
  // partition padded to 8-row groups, groups stored in the K-major
  // core-matrix layout of tc.cuh (K = tc_kp, a multiple of 32 bytes)
  void* tc_rows = nullptr;        // [tc_groups * 8 * tc_kp] elements of dtype
  int64_t* tc_gstart = nullptr;   // [c + 1] first group of each partition
  int32_t* tc_ids = nullptr;      // [tc_groups * 8] point id (-1 on padding)
  float* tc_norms = nullptr;      // [tc_groups * 8] ||x|| (0 on padding)
  float* tc_pmax = nullptr;       // [c] largest ||x|| of each partition
  int32_t tc_kp = 0;
  int64_t tc_groups = 0;
  int32_t* assign = nullptr;      // [n][1 + spills] copy of the assignment
  // codebook packed for the tensor-core partition selection (select_tc.cu):
  // tiles of 64 centroids, each the tf32 hi part then the lo part in the
  // core-matrix layout (K = sel_kp); null when that kernel does not apply
  float* sel_cb = nullptr;
  int32_t sel_kp = 0, sel_tiles = 0;
  // PQ4 indexes: codebooks [pq_m][16][2] of the residuals; the codes of every
  // copy are `vectors` ([rows][code_stride] bytes, two 4-bit codes a byte)
  float* pq_cb = nullptr;
  int32_t pq_m = 0;
};

}  // namespace soar

// The opaque handle of the C ABI.
struct soar_index {
  soar::IndexData data;
};

namespace soar {

void build_index(IndexData& ix, const void* X, soar_dtype dt, const float* C, const int32_t* assign,
                 cudaStream_t s, const float* pq_cb = nullptr);

// PQ codebooks B [d/2][16][2] of the residuals X[i] - C[part[i]] (pq.cu).
void pq_train(const void* X, soar_dtype dt, int64_t n, int32_t d, const float* C, const int32_t* part,
              int32_t iters, const int32_t* init_idx, float* B, cudaStream_t s, Scratch& scr);
// Codes of every index row from its residual x - C_p (pq.cu).
void pq_encode_index(IndexData& ix, const void* X, soar_dtype dt, cudaStream_t s, Scratch& scr);
void free_index(IndexData& ix);

// A flat index over fx.n rows (fx.vectors, fx.dtype, fx.row_stride, fx.d and
// fx.c = ceil(n / chunk) set by the caller; chunk a multiple of 8): chunk p
// holds rows [p * chunk, (p + 1) * chunk) with their ids, plus the
// tensor-core layout of the rows; every array is taken from `scr`.  Lets the
// partition scan serve as an exact brute force.
void build_flat_tc(IndexData& fx, int64_t chunk, cudaStream_t s, Scratch& scr);

// index_io.cu: the index's device arrays to / from a file (format in index_io.cu).
void save_index(const IndexData& ix, const char* path, cudaStream_t s);
void load_index(IndexData& ix, const char* path, cudaStream_t s);

void quantize_fp8(const void* V, soar_dtype dt, int64_t m, int32_t d, uint8_t* codes,
                  int32_t code_stride, float* scales, cudaStream_t s);

// ----------------------------------------------------------- select_tc.cu

// Whether the packed selection codebook of K = kp columns fits the kernel.
bool select_tc_fits(int kp);
// Fills out [sel_tiles][2][64 * sel_kp] from ix.centroids.
void pack_select_codebook(const IndexData& ix, float* out, cudaStream_t s);
// Whether select_tc takes these queries (packed codebook present, t <= 32,
// rows 16-byte aligned).
bool select_tc_usable(const IndexData& ix, const float* Qf, int qstride, int t);
// top [nq][t] (and top_s, if not null): each query's t best centroids by
// inner product, best first, lower id on ties; fp32 queries Qf [nq][qstride].
void select_tc(const IndexData& ix, const float* Qf, int64_t nq, int qstride, int t, int32_t* top, float* top_s,
               cudaStream_t s);

// ----------------------------------------------------------- search.cu

void select_partitions(const IndexData& ix, const void* Q, soar_dtype dt, int64_t nq, int32_t t,
                       int32_t* top, float* top_scores, cudaStream_t s, Scratch& scr);
// S [nq][c] = the centroid scores the search ranks partitions by.
void centroid_scores(const IndexData& ix, const void* Q, soar_dtype dt, int64_t nq, float* S, cudaStream_t s,
                     Scratch& scr);

// ----------------------------------------------------------- mlp.cu
int64_t mlp_param_count(int D, int H);
void mlp_forward(const float* P, int D, int H, const float* Z, int B, bool bf16, float* A1, float* H1, float* A2,
                 float* H2, float* y, cudaStream_t s);
void mlp_backward(const float* P, int D, int H, const float* Z, const float* target, int B, bool bf16, float* G,
                  float* loss, cudaStream_t s, Scratch& scr);
void mlp_adam(float* P, const float* G, float* m1, float* m2, int64_t n, int step, float lr, float b1, float b2,
              float eps, cudaStream_t s);
void mlp_predict(const float* P, int D, int H, const float* Z, int B, bool bf16, float alpha, int c, float* y_out,
                 int32_t* t_out, cudaStream_t s, Scratch& scr);
void probe_features(const IndexData& ix, const void* Q, soar_dtype dt, int64_t nq, int top, float* Z,
                    cudaStream_t s, Scratch& scr);
void probe_labels(const IndexData& ix, const void* Q, soar_dtype dt, int64_t nq, const int64_t* truth, int k,
                  float target, int32_t* labels, cudaStream_t s, Scratch& scr);
// Z [nq][d + top] = [q || top_s] (the probe features, from scores already selected).
void features_from_scores(const void* Q, soar_dtype dt, int64_t nq, int d, const float* top_s, int top, float* Z,
                          cudaStream_t s);

// The learned probe count inside a search: the search's own top-t selection
// (with scores) gives the features, the network predicts each query's probe
// count, clamp(ceil(alpha exp(y)), 1, t_cap), and the query probes that many
// of its top-t partitions.  t_out (nullable) receives the counts.
struct LearnedProbe {
  const float* params;
  int d_in, hidden;
  bool bf16;
  float alpha;
  int t_cap;
  int32_t* t_out;
};

// Same computation as select_partitions with all scratch carved from a
// caller-provided device buffer of select_scratch_bytes(ix, nq) bytes.
size_t select_scratch_bytes(const IndexData& ix, int64_t nq);
void select_partitions_in(const IndexData& ix, const void* Q, soar_dtype dt, int64_t nq, int32_t t, int32_t* top,
                          float* top_scores, void* scratch, cudaStream_t s);

// With `coarse` set, the probed partitions come from multilevel_select
// (t1 coarse probes) instead of the flat top-t selection.
// With `learned` set, the per-query probe counts come from the network.
void search(const IndexData& ix, const void* Q, soar_dtype dt, int64_t nq, int32_t k, int32_t t,
            const int32_t* t_per_query, int32_t rescore, int64_t* ids_out, float* scores_out,
            cudaStream_t s, Scratch& scr, const IndexData* coarse = nullptr, int32_t t1 = 0,
            const LearnedProbe* learned = nullptr);

// Two-level partition selection: an IVF search over the fine centroids (the
// rows of `coarse`) with t1 coarse probes and k = t.  top [nq][t] fine
// partition ids, best first, -1 after the last one found; count [nq] the
// number found; top_scores [nq][t] (nullable) their <q, C_i>.
void multilevel_select(const IndexData& coarse, const void* Q, soar_dtype dt, int64_t nq, int32_t t, int32_t t1,
                       int32_t* top, float* top_scores, int32_t* count, cudaStream_t s, Scratch& scr);

void merge_topk(const int64_t* ids, const float* scores, int64_t nq, int m, int len, const int64_t* id_offsets,
                int k, int64_t* ids_out, float* scores_out, cudaStream_t s, Scratch& scr);

void exact_mips(const void* X, soar_dtype xdt, int64_t n, int32_t d, const void* Q, soar_dtype qdt,
                int64_t nq, int32_t k, int64_t* ids_out, float* scores_out, cudaStream_t s,
                Scratch& scr);

}  // namespace soar
