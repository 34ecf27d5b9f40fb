/*
 * soar.h -- C ABI of the GB300 (sm_103a) SOAR spilled-IVF library.
 *
 * SOAR ("Spilling with Orthogonality-Amplified Residuals", Sun et al.,
 * arXiv 2404.00774) builds an inverted-file (IVF) index over a codebook C
 * of c centroids and assigns every datapoint x to its nearest centroid
 * pi(x) plus `spills` further centroids chosen by the loss of Theorem 3.1,
 *     ||x - c'||^2 + lambda * <x - c', r_hat>^2,   r_hat = (x - C[pi(x)]) / ||x - C[pi(x)]||.
 * Search (Section 2.2) ranks the centroids by <q, C_i>, scans the top t
 * partitions, removes the duplicate copies that spilling creates
 * (Section 3.5) and returns the top k by <q, x> (maximum inner product,
 * Section 2.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Array arguments are DEVICE pointers owned by the caller unless a
 *   comment says "host".  Matrices are dense row-major; a vector set
 *   X[n][d] has row stride d elements.  Rows must be 4-byte aligned;
 *   16-byte aligned rows (d*elem_size a multiple of 16) take faster loads.
 * - `stream` orders the call's device work; calls return as soon as the
 *   work is queued unless documented otherwise.  The caller synchronises.
 *   Scratch memory is taken from the device's stream-ordered pool
 *   (cudaMallocAsync on `stream`) and released in stream order.
 * - Every call returns a soar_status and never throws across the ABI.
 *   Argument errors return SOAR_EINVAL before any device work is queued
 *   and leave outputs untouched.  soar_last_error() gives a thread-local
 *   message for the last failing call on the calling thread.
 * - Tie rules: an argmin over centroids prefers the lower centroid index;
 *   top-t partitions and top-k results are ordered by score descending,
 *   the lower id first on equal scores.  Fewer than k distinct candidates
 *   leave id -1 and score -inf in the tail.
 * - Errors raised by kernels after the call returned surface at the next
 *   synchronising CUDA call as SOAR_ECUDA.
 */
#ifndef SOAR_H
#define SOAR_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#if defined(__GNUC__)
#define SOAR_API __attribute__((visibility("default")))
#else
#define SOAR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SOAR_OK = 0,
  SOAR_EINVAL = 1,        /* invalid argument (sizes, null pointers, NaN lambda ...) */
  SOAR_ENOMEM = 2,        /* device allocation failed */
  SOAR_ECUDA = 3,         /* a CUDA runtime error (message in soar_last_error) */
  SOAR_ETIMEOUT = 4,      /* a bounded device wait ran out */
  SOAR_EUNSUPPORTED = 5   /* valid but outside what this build implements */
} soar_status;

/* Element type of caller-provided vector sets (datapoints, queries). */
typedef enum { SOAR_F32 = 0, SOAR_BF16 = 1 } soar_dtype;

/* How an index scores candidates during search.
 * SOAR_SCORE_F32: duplicated rows are stored in the input dtype and scored
 *   exactly (fp32 products and sums).
 * SOAR_SCORE_FP8: duplicated rows are FP8-E4M3 codes with one fp32 scale
 *   per row (scale = max|row| / 448); queries and centroids are scored the
 *   same way; a single copy of the original vectors, indexed by id, serves
 *   the exact fp32 rescoring of the best `rescore` candidates.  This is the
 *   GPU analogue of the paper's layout in Section 3.5: only the compressed
 *   representation is duplicated, the highest-bitrate copy is stored once.
 * SOAR_SCORE_PQ4: every copy holds a 4-bit product-quantization code of its
 *   partitioning residual x - C_p (2 dimensions and 16 centres per subspace,
 *   Section 3.5 and App. A.3); the approximate score of a copy is
 *   <q, C_p> + sum_s <q_s, B_s[code_s]>; the original vectors are stored once
 *   and rescore the best `rescore` candidates exactly.  Built with
 *   soar_index_build_pq.
 */
/* (Value 1 is unused: bf16 storage comes from the input dtype.  An index
 * built from SOAR_BF16 data with SOAR_SCORE_F32 keeps the bf16 rows, screens
 * them on the tensor cores and scores them exactly.) */
typedef enum { SOAR_SCORE_F32 = 0, SOAR_SCORE_FP8 = 2, SOAR_SCORE_PQ4 = 3 } soar_score_mode;

typedef struct soar_index soar_index;   /* opaque; owns its device memory */

/* Thread-local message of the last failing call ("" if none). */
SOAR_API const char* soar_last_error(void);

/* Library version string, e.g. "soar-gb300 0.1 sm_103a". */
SOAR_API const char* soar_version(void);

/*
 * Lloyd k-means (Section 2.2: "Vector quantization" trains the codebook C).
 *   X        [n][d] datapoints (dtype)
 *   init_idx [c]    distinct row indices of X used as the initial centroids
 *                   (the caller draws them; the library draws no random numbers)
 *   C_out    [c][d] fp32 output codebook
 * Each of `iters` iterations assigns every point to its nearest centroid
 * (ties to the lower index) and replaces every non-empty centroid by the
 * mean of its points, summed in fp64 and rounded to fp32; an empty cluster
 * keeps its previous centroid.  Requires 1 <= c <= n, iters >= 0, d >= 1;
 * init_idx entries outside [0, n) give SOAR_EINVAL (checked on the device,
 * which costs one synchronisation of `stream`).
 */
SOAR_API soar_status soar_train_centroids(const void* X, soar_dtype dtype, int64_t n, int32_t d,
                                 int32_t c, int32_t iters, const int32_t* init_idx,
                                 float* C_out, cudaStream_t stream);

/*
 * Primary and SOAR spilled assignment (Section 2.2 for pi; Eq. 2 and
 * Theorem 3.1 for the spills; Section 3.5 for the order of the pipeline).
 *   X          [n][d] datapoints (dtype)
 *   C          [c][d] fp32 codebook
 *   assign_out [n][1 + spills] int32: column 0 is pi(x) = argmin ||x - C_i||^2,
 *              column j >= 1 is the j-th spilled partition, the argmin over
 *              centroids not yet assigned to x of
 *                  ||x - c'||^2 + lambda * sum_{i<j} <x - c', r_hat_i>^2,
 *              r_hat_i the unit residual of the i-th earlier assignment
 *              (j = 1 is exactly the paper's loss; a zero residual adds no
 *              penalty).  lambda = 0 gives plain nearest-centroid spilling.
 * Requires lambda finite and >= 0, 0 <= spills <= 4, c >= 1 + spills.
 */
SOAR_API soar_status soar_assign(const void* X, soar_dtype dtype, int64_t n, int32_t d,
                        const float* C, int32_t c, float lambda, int32_t spills,
                        int32_t* assign_out, cudaStream_t stream);

/*
 * Inverted-file index over a codebook and an assignment (Section 2.2,
 * Section 3.5).  Partition p lists, in ascending id, every point with p in
 * its assignment row; each listed point's vector is copied next to its id
 * so a partition is one contiguous block of rows.
 *   X      [n][d] datapoints (dtype); copied, the caller may free it after the call
 *   C      [c][d] fp32 codebook; copied
 *   assign [n][1 + spills] int32 (as produced by soar_assign)
 *   out    host pointer that receives the new index handle
 * This call synchronises `stream` once (to size the index) and returns
 * after the index is complete.  Every assignment must lie in [0, c) and the
 * entries of a row must be distinct (checked; SOAR_EINVAL otherwise).
 */
SOAR_API soar_status soar_index_build(const void* X, soar_dtype dtype, int64_t n, int32_t d,
                             const float* C, int32_t c, const int32_t* assign, int32_t spills,
                             soar_score_mode mode, soar_index** out, cudaStream_t stream);

/* Read-only description of an index (all pointers are device pointers owned by the index). */
typedef struct {
  int64_t n;               /* datapoints */
  int32_t d;               /* dimension */
  int32_t c;               /* partitions */
  int32_t spills;          /* extra assignments per point */
  int32_t mode;            /* soar_score_mode */
  int32_t dtype;           /* soar_dtype of the stored vectors */
  int32_t row_stride;      /* elements per stored row (>= d, padded for 16-byte rows) */
  int64_t rows;            /* n * (1 + spills) */
  int64_t max_partition;   /* largest partition size */
  const int64_t* offsets;  /* [c + 1] partition p is rows offsets[p] .. offsets[p+1]-1 */
  const int32_t* ids;      /* [rows] point id of each row */
  const void* vectors;     /* [rows][row_stride] dtype (SOAR_SCORE_F32) or FP8 codes (SOAR_SCORE_FP8) */
  const float* row_scales; /* [rows] per-row FP8 scale (SOAR_SCORE_FP8) or NULL */
  const void* originals;   /* [n][row_stride] single copy for rescoring (SOAR_SCORE_FP8) or NULL */
  const float* centroids;  /* [c][d] fp32 */
  int64_t device_bytes;    /* device memory held by the index */
} soar_index_info;

SOAR_API soar_status soar_index_get_info(const soar_index* index, soar_index_info* info /* host */);

/* Frees the index and its device memory (after synchronising the device work that used it). */
SOAR_API soar_status soar_index_free(soar_index* index);

/*
 * Index persistence, so that a large index (the inverted lists of Section 2.2
 * with the spilled copies of Section 3.5) is built once and reused.
 * soar_index_save writes every device array of the index, after a fixed
 * header (magic "SOARIDX1", format version 2, the scalar fields, the byte
 * size of each array), to the file `path` (host string; an existing file is
 * replaced).  soar_index_load reads such a file into a new index on the
 * current device; its searches return what the saved index returned, bit
 * for bit.  Both move the data through a pinned host buffer of 64 MiB with
 * one copy per chunk on `stream`, and synchronise `stream`; both return after
 * the file is complete.  A file that is not a SOAR index, has header fields
 * out of range, a section of the wrong size, a required section missing, or
 * is shorter or longer than its header says gives SOAR_EINVAL; another format
 * version gives SOAR_EUNSUPPORTED.  All of these are found on the host,
 * before any device memory is taken.
 */
SOAR_API soar_status soar_index_save(const soar_index* index, const char* path, cudaStream_t stream);
SOAR_API soar_status soar_index_load(const char* path, soar_index** out /* host */, cudaStream_t stream);

/*
 * Top-t partitions per query: MIPS_t(q, C) (Section 2.2), the centroids of
 * largest <q, C_i>, in rank order.
 *   Q         [nq][d] queries (dtype)
 *   top_out   [nq][t] int32 partition ids
 *   score_out [nq][t] fp32 scores, may be NULL
 * Scores are fp32 (SOAR_SCORE_F32 indices) or FP8-scaled (SOAR_SCORE_FP8).
 * Ties go to the lower partition id.  For t <= 32 on fp32 centroids with d <= 104
 * the scores come from the tensor cores with each fp32 value split into two
 * tf32 parts (three products), an error within that of a fp32 dot product;
 * otherwise from a fp32 GEMM.  Requires 1 <= t <= min(c, 8192).
 */
SOAR_API soar_status soar_select_partitions(const soar_index* index, const void* Q, soar_dtype dtype,
                                   int64_t nq, int32_t t, int32_t* top_out, float* score_out,
                                   cudaStream_t stream);

/*
 * IVF search with deduplication of spilled copies (Section 2.2, Section 3.5).
 *   Q           [nq][d] queries (dtype)
 *   t           partitions probed per query (1 <= t <= min(c, 8192))
 *   t_per_query [nq] int32 per-query probe counts in [0, t] (values outside are
 *               clamped; 0 probes nothing and gives only padding), or NULL for t everywhere
 *   rescore     SOAR_SCORE_FP8 and SOAR_SCORE_PQ4 indices: candidates kept per query
 *               (the best approximate scores of the probed union, each point once)
 *               for exact fp32 rescoring (k <= rescore <= 4096); ignored (pass 0)
 *               for SOAR_SCORE_F32
 *   ids_out     [nq][k] int64 point ids, scores_out [nq][k] fp32 <q, x>
 * Requires 1 <= k <= 1024.
 */
SOAR_API soar_status soar_search(const soar_index* index, const void* Q, soar_dtype dtype, int64_t nq,
                        int32_t k, int32_t t, const int32_t* t_per_query, int32_t rescore,
                        int64_t* ids_out, float* scores_out, cudaStream_t stream);

/* ------------------------------------------------------------------ *
 * Multi-level VQ (App. A.4, general index setup; Section 4).  The fine
 * centroids of an index (c of them, often millions) are vector-quantized
 * again into c2 coarse partitions, with SOAR spilling at that level too
 * (the multiple assignments happen at each level of the tree).  The coarse
 * level is an ordinary soar_index whose n = c rows are the fine centroids
 * (fp32, mode SOAR_SCORE_F32), so partition selection (S = Q C^T, top t,
 * Section 2.2) becomes an IVF search over the centroids: probe the t1
 * coarse partitions of largest <q, C2_j>, take the union of their fine
 * centroids (a spilled one counts once) and keep the t of largest <q, C_i>
 * (score descending, lower id first on ties).  When the probed coarse
 * partitions hold fewer than t fine centroids the query probes only those.
 * ------------------------------------------------------------------ */

/* Builds the coarse index of `index` (the second VQ level of App. A.4):
 * k-means over its c fine centroids
 * (c2 clusters, `iters` Lloyd steps from the rows init_idx [c2] (device
 * int32, distinct, in [0, c)), fp64 update as soar_train_centroids), then
 * the primary and `spills` SOAR assignments with weight `lambda` (as
 * soar_assign), then soar_index_build over those rows.  The fine index is
 * only read.  *out owns its own device memory (free with soar_index_free).
 * Requires 1 + spills <= c2 <= c, 0 <= spills <= 4, lambda finite >= 0. */
SOAR_API soar_status soar_index_build_coarse(const soar_index* index, int32_t c2, int32_t iters,
                                             const int32_t* init_idx, float lambda, int32_t spills,
                                             soar_index** out, cudaStream_t stream);

/* The two-level selection alone (App. A.4: partition selection as an IVF
 * search over the centroids).
 *   coarse    a coarse index (rows = the fine centroids, fp32)
 *   Q         [nq][d] queries (dtype), device
 *   t, t1     fine partitions kept (1 <= t <= min(c, 1024)), coarse partitions
 *             probed (1 <= t1 <= min(c2, 8192))
 *   top_out   [nq][t] int32 fine partition ids, best first, -1 after the last found
 *   score_out [nq][t] fp32 <q, C_i> (-inf on padding), or NULL
 *   count_out [nq] int32 number of fine partitions found (0 when every probed
 *             coarse partition is empty) */
SOAR_API soar_status soar_select_partitions_multilevel(const soar_index* coarse, const void* Q, soar_dtype dtype,
                                                       int64_t nq, int32_t t, int32_t t1, int32_t* top_out,
                                                       float* score_out, int32_t* count_out, cudaStream_t stream);

/* soar_search (Section 2.2, Section 3.5) with the probed partitions chosen
 * by the two-level selection of App. A.4:
 * the query probes the fine partitions soar_select_partitions_multilevel
 * returns (fewer than t when fewer were found; none gives only padding).
 * `coarse` must be a coarse index of `index` (n == index's c, same d, fp32).
 * Other arguments and results as soar_search (t <= min(c, 1024)). */
SOAR_API soar_status soar_search_multilevel(const soar_index* index, const soar_index* coarse, const void* Q,
                                            soar_dtype dtype, int64_t nq, int32_t k, int32_t t, int32_t t1,
                                            int32_t rescore, int64_t* ids_out, float* scores_out,
                                            cudaStream_t stream);

/*
 * Merge of m result lists per query into one top k (the exchange step of a
 * search whose rows are sharded over several GPUs: every shard searches its
 * own rows under the same codebook, so it probes the same partitions, and
 * the per-shard top k lists are merged; Section 3.5's rule that a point
 * counts once applies across the lists).
 *   ids, scores  [nq][m][len] int64 / fp32, each list best first, id -1 (score
 *                -inf) closing a shorter list, as soar_search writes them
 *   id_offsets   [m] int64 added to the ids of list j (a shard's first global
 *                row), or NULL for none
 *   ids_out, scores_out [nq][k]: the k best by score desc, lower id first on
 *                ties; an entry equal in id and score to the one before it is
 *                dropped; -1 / -inf padding.
 * Requires 1 <= m <= 4096, 1 <= len <= 1024, 1 <= k <= 1024, offset ids < 2^31.
 */
SOAR_API soar_status soar_merge_topk(const int64_t* ids, const float* scores, int64_t nq, int32_t m, int32_t len,
                                     const int64_t* id_offsets, int32_t k, int64_t* ids_out, float* scores_out,
                                     cudaStream_t stream);

/*
 * Exact maximum inner product search MIPS_k(q, X) (Section 2.1) by brute
 * force: fp32 products and sums over every datapoint.
 *   X [n][d] (xdtype), Q [nq][d] (qdtype), ids_out [nq][k] int64, scores_out [nq][k] fp32.
 * Requires 1 <= k <= 1024.
 */
SOAR_API soar_status soar_exact_mips(const void* X, soar_dtype xdtype, int64_t n, int32_t d,
                            const void* Q, soar_dtype qdtype, int64_t nq, int32_t k,
                            int64_t* ids_out, float* scores_out, cudaStream_t stream);

/*
 * Product-quantization codebooks of the partitioning residuals (Section
 * 3.5, App. A.3): r = x - C[part[i]] formed in fp32 for the n training rows,
 * then for every subspace s (dimensions 2s and 2s+1) Lloyd's k-means with 16
 * centres started from the rows init_idx [16] (distinct, in [0, n), device
 * int32; the same rows for every subspace), `iters` steps, each centre the
 * fp64 mean of its rows rounded to fp32 (an empty one keeps its value).
 *   X [n][d] (dtype), C [c][d] fp32, part [n] int32 in [0, c) (each row's
 *   primary partition), B_out [d/2][16][2] fp32.  Requires d even.
 */
SOAR_API soar_status soar_pq_train(const void* X, soar_dtype dtype, int64_t n, int32_t d, const float* C, int32_t c,
                                   const int32_t* part, int32_t iters, const int32_t* init_idx, float* B_out,
                                   cudaStream_t stream);

/*
 * soar_index_build with mode SOAR_SCORE_PQ4 (Section 3.5 and App. A.3: only
 * the compressed codes are duplicated): every copy (point x in
 * partition p) is encoded from x - C_p with the codebooks B [d/2][16][2]
 * (per subspace the nearest centre, the lower index on ties), two codes per
 * byte (the even subspace in the low nibble); the original vectors are
 * stored once, indexed by id.  Other arguments as soar_index_build.
 */
SOAR_API soar_status soar_index_build_pq(const void* X, soar_dtype dtype, int64_t n, int32_t d, const float* C,
                                         int32_t c, const int32_t* assign, int32_t spills, const float* B,
                                         soar_index** out, cudaStream_t stream);

/*
 * Per-row FP8-E4M3 quantisation used by SOAR_SCORE_FP8 indices (the
 * compressed, duplicated form of the Section 3.5 layout analogue):
 * scale[i] = max_j |V[i][j]| / 448 (1 when the row is zero) and
 * codes[i][j] = e4m3(V[i][j] / scale[i]) rounded to nearest-even and
 * saturated to +-448.  Exposed so the codes can be checked bit for bit.
 *   V [m][d] (dtype), codes [m][code_stride] uint8 (code_stride >= d), scales [m] fp32.
 */
SOAR_API soar_status soar_quantize_fp8(const void* V, soar_dtype dtype, int64_t m, int32_t d,
                              uint8_t* codes, int32_t code_stride, float* scales,
                              cudaStream_t stream);

/*
 * soar_select_partitions_static: soar_select_partitions without any device
 * allocation.  The paper has no counterpart; this exists for callers that
 * must not allocate device memory at call time -- for example a host
 * framework that owns the whole device memory budget and forbids other
 * allocators, or a latency-critical serving thread that must never enter
 * the CUDA allocator (cudaMalloc / cudaFree can block on the device and on
 * the driver's locks).  Same arguments and results as
 * soar_select_partitions.
 *
 * Scratch (the queries' padded rows and the nq x c score matrix, at most
 * SOAR_STATIC_SCRATCH_BYTES; the limit is checked on that size even when the
 * tensor-core selection needs no score matrix) lives in a fixed device array inside this
 * library: every GPU that loads the library holds those bytes until the
 * process exits.  A batch that needs more returns SOAR_EINVAL with the
 * byte count in soar_last_error(); split it into smaller calls.  The first
 * call on each device (with that device current) looks the array's device
 * address up once; make that first call before any stream capture.
 * All calls on one device share the array and every call overwrites what it
 * reads, so calls that overlap on the GPU (different streams, or host
 * threads without ordering between them) race and must be serialised by the
 * caller, e.g. by issuing them on one stream.
 */
#define SOAR_STATIC_SCRATCH_BYTES (32u << 20)
SOAR_API soar_status soar_select_partitions_static(const soar_index* index, const void* Q, soar_dtype dtype,
                                                   int64_t nq, int32_t t, int32_t* top_out, float* score_out,
                                                   cudaStream_t stream);

/* ------------------------------------------------------------------ *
 * Learned probe count (an extension; the paper has no counterpart)
 * ------------------------------------------------------------------ *
 * A small MLP predicts, per query, how many partitions to probe.  Input
 * z(q) = [q || the query's top-`top` centroid scores, descending]
 * (d_in = d + top); two hidden layers of `hidden` units with ReLU; one
 * output y, trained by mean squared error against log t*(q).  Parameters are
 * one fp32 device buffer of soar_mlp_param_count(d_in, hidden) values laid
 * out W1 [hidden][d_in] | b1 [hidden] | W2 [hidden][hidden] | b2 [hidden] |
 * W3 [hidden] | b3 [1] (row-major); the caller initialises it.  With bf16 != 0
 * every product rounds its operands to bf16 and accumulates in fp32.
 */
SOAR_API int64_t soar_mlp_param_count(int32_t d_in, int32_t hidden);

/* Z_out [nq][d + top] fp32 features z(q) above (an extension): the query,
 * then its top-`top` centroid scores <q, C_i> of Section 2.2, descending
 * (top <= min(c, 8192)). */
SOAR_API soar_status soar_probe_features(const soar_index* index, const void* Q, soar_dtype dtype, int64_t nq,
                                         int32_t top, float* Z_out, cudaStream_t stream);

/* labels_out [nq] int32 (an extension; recall@k of Section 2.1, probe order of
 * Section 2.2): t*(q), the smallest probe count whose recall@k reaches
 * target_recall, given the query's exact top-k `truth_ids` [nq][k] (int64,
 * e.g. from soar_exact_mips).  A neighbour is found at probe count t when one
 * of its partitions has position <= t in the query's probe order (ties to the
 * lower id); t* is the ceil(target_recall * k)-th smallest such position. */
SOAR_API soar_status soar_probe_labels(const soar_index* index, const void* Q, soar_dtype dtype, int64_t nq,
                                       const int64_t* truth_ids, int32_t k, float target_recall,
                                       int32_t* labels_out, cudaStream_t stream);

/* y_out [batch] = network output for Z [batch][d_in] (the MLP above, an
 * extension). */
SOAR_API soar_status soar_mlp_forward(const float* params, int32_t d_in, int32_t hidden, const float* Z,
                                      int32_t batch, int32_t bf16, float* y_out, cudaStream_t stream);

/* The MLP above (an extension): grads_out (same layout as params) =
 * d/dparams of mean((y - target)^2) over
 * the batch; loss_out (device float, may be NULL) = that loss. */
SOAR_API soar_status soar_mlp_backward(const float* params, int32_t d_in, int32_t hidden, const float* Z,
                                       const float* target, int32_t batch, int32_t bf16, float* grads_out,
                                       float* loss_out, cudaStream_t stream);

/* Training the MLP above (an extension): one Adam step (bias-corrected, step
 * counted from 1) on `count` parameters;
 * m1, m2 are the caller's moment buffers (start at zero). */
SOAR_API soar_status soar_mlp_adam(float* params, const float* grads, float* m1, float* m2, int64_t count,
                                   int32_t step, float lr, float beta1, float beta2, float eps,
                                   cudaStream_t stream);

/* The MLP above (an extension): t_out [batch] = clamp(ceil(alpha * exp(y)),
 * 1, c), per-query probe counts
 * for soar_search's t_per_query. */
SOAR_API soar_status soar_mlp_predict_probes(const float* params, int32_t d_in, int32_t hidden, const float* Z,
                                             int32_t batch, int32_t bf16, float alpha, int32_t c, int32_t* t_out,
                                             cudaStream_t stream);

/* soar_search with the learned probe count in one call: the search selects
 * each query's top `top` partitions with their scores (the selection of
 * soar_probe_features, done once), the network predicts the query's count
 * clamp(ceil(alpha * exp(y)), 1, t_cap) from those features, and the query
 * probes that many of its top partitions, best first.  The results equal
 * soar_search(index, Q, ..., t = top, t_per_query = those counts).
 *   params, hidden, bf16   the network (d_in = d + top), as soar_mlp_forward
 *   t_out                  [nq] int32 device, the counts used (nullable)
 *   rescore, ids_out, scores_out as soar_search.
 * Requires 1 <= t_cap <= top <= min(c, 8192), alpha finite and > 0; the
 * fastest path takes top <= 32 (the selection kernel of Section 2.2 keeps up
 * to 32 partitions per query in registers). */
SOAR_API soar_status soar_search_learned(const soar_index* index, const void* Q, soar_dtype dtype, int64_t nq,
                                         int32_t k, int32_t top, const float* params, int32_t hidden, int32_t bf16,
                                         float alpha, int32_t t_cap, int32_t rescore, int64_t* ids_out,
                                         float* scores_out, int32_t* t_out, cudaStream_t stream);

/* ------------------------------------------------------------------ *
 * Serving loop (an extension; the paper describes no serving system)
 * ------------------------------------------------------------------ *
 * Continuous batching over a resident SOAR_SCORE_F32 index.  Requests (one
 * fp32 host query of d values, its own k and t) are queued from any thread;
 * a dispatcher thread keeps up to `streams` batches in flight, each on its own
 * CUDA stream.  Whenever a stream slot is free it forms the next batch from
 * the pending requests in arrival order, admitting requests while the batch
 * holds at most max_batch queries and the estimated device scratch of all
 * batches in flight stays within memory_budget bytes (a request alone is
 * always admitted when nothing runs) and holds requests of one k class
 * (k <= 32 or k > 32; the other class keeps its place in the queue).  A batch
 * is one soar_search with per-request probe counts and the batch's largest k;
 * each request receives its own top k.  The index must outlive the server.
 */
typedef struct {
  int32_t max_batch;       /* queries per batch, 1..4096 */
  int32_t streams;         /* batches in flight, 1..16 */
  int64_t memory_budget;   /* bytes of device scratch admitted in flight */
  int32_t max_k;           /* largest k a request may ask for, 1..1024 */
} soar_server_config;

typedef struct {
  uint64_t batches;            /* batches launched */
  uint64_t completed;          /* requests completed */
  uint64_t queries_in_batches; /* requests launched (sum of batch sizes) */
  uint64_t pending;            /* requests waiting for a batch */
  int32_t max_in_flight;       /* most batches seen on the GPU at once */
  double p50_ms, p99_ms;       /* request latency (submit to results on the host) */
} soar_server_metrics;

typedef struct soar_server soar_server;

SOAR_API soar_status soar_server_create(const soar_index* index, const soar_server_config* cfg,
                                        soar_server** out /* host */);
/* query: host [d] fp32 (copied); request_id: host out.  1 <= k <= max_k, 1 <= t <= min(c, 8192). */
SOAR_API soar_status soar_server_submit(soar_server* server, const float* query, int32_t k, int32_t t,
                                        uint64_t* request_id);
/* Queues n requests at once: queries host [n][d] fp32 (copied), ks / ts host
 * [n] (limits as for soar_server_submit), request_ids host out [n].
 * arrival_s (host [n], may be NULL): each request's arrival time in seconds
 * after this call (0 <= arrival_s < 1e6); a request joins the pending queue
 * when its time comes and its latency counts from then (an open-loop replay
 * of an arrival trace).  NULL: all arrive now.  Any invalid entry rejects the
 * whole call (SOAR_EINVAL) before anything is queued. */
SOAR_API soar_status soar_server_submit_many(soar_server* server, const float* queries, int64_t n, const int32_t* ks,
                                             const int32_t* ts, const double* arrival_s, uint64_t* request_ids);
/* Collects n requests in order (each once): ids_out / scores_out host
 * [n][kstride] receive each request's own k results, the rest of the row
 * padded with -1 / -inf; latency_ms host [n] may be NULL.  timeout_ms bounds
 * the whole call (SOAR_ETIMEOUT).  Returns the last failing request status,
 * else SOAR_OK. */
SOAR_API soar_status soar_server_wait_many(soar_server* server, const uint64_t* request_ids, int64_t n,
                                           int32_t kstride, int64_t* ids_out, float* scores_out, double* latency_ms,
                                           int32_t timeout_ms);
/* Blocks until the request completed (or timeout_ms passed: SOAR_ETIMEOUT) and
 * copies its k ids / scores to host memory; latency_ms (may be NULL) receives
 * submit-to-completion time.  Each request can be collected once. */
SOAR_API soar_status soar_server_wait(soar_server* server, uint64_t request_id, int64_t* ids_out, float* scores_out,
                                      double* latency_ms, int32_t timeout_ms);
SOAR_API soar_status soar_server_stats(soar_server* server, soar_server_metrics* out /* host */);
/* Finishes the queued requests, stops the dispatcher and frees the server. */
SOAR_API soar_status soar_server_destroy(soar_server* server);

/*
 * Synchronises the current device and reports device-side failures of
 * earlier calls: SOAR_ETIMEOUT when a kernel gave up one of its bounded
 * waits (its results are incomplete), SOAR_ECUDA for a CUDA error.  Clears
 * the recorded failure.
 */
SOAR_API soar_status soar_check_device(void);

/* ------------------------------------------------------------------ *
 * Instrumentation (measurement support; not part of the paper's method)
 * ------------------------------------------------------------------ */

/* Number of CUDA kernels this library has launched in this process. */
SOAR_API uint64_t soar_kernel_launches(void);

/* Longest wait, in SM clock cycles, of the partition scan's pipeline (a
 * copy landing, an accumulator filling or freeing) before the waiting CTA
 * gives up: it then records the failure for soar_check_device, stops taking
 * work, lets its copies and MMAs in flight land (those waits keep the default
 * of about 2^31 cycles) and frees its tensor memory, and the finishing of that
 * search reads its unwritten lists as empty.  0 restores the default.  Applies
 * to the scans launched after the call; a test of the failure path, not a
 * tuning knob. */
SOAR_API soar_status soar_set_wait_limit(int64_t cycles);

/* Turns on (1) or off (0) CUDA-event timing of the named stages of
 * soar_search ("select", "group", "scan", "merge", "rescore"); events are
 * recorded on the call's stream around each stage, adding no synchronisation. */
SOAR_API soar_status soar_stage_timing(int enable);

/* Waits for the recorded events, writes the total milliseconds and the
 * number of timed launches per stage since the last read, and clears them.
 * `names` (host, names_len bytes) receives the comma-separated stage names
 * in the order of `ms` / `launches` (host arrays of max_stages entries).
 * Returns the number of stages written. */
SOAR_API int soar_stage_times(char* names, int names_len, float* ms, int* launches, int max_stages);

#ifdef __cplusplus
}
#endif

#endif /* SOAR_H */
