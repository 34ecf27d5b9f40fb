// Types shared by the partition-scan kernels (SIMT and tensor-core).
#pragma once

#include "internal.cuh"

namespace soar {

// One candidate of a per-query top-k list.
struct Cand {
  float s;
  int32_t id;
};

// Order of the top-k lists: higher score first, lower id first on ties
// (id -1, the empty slot, loses every tie).
__device__ __forceinline__ bool better(float a, int ia, float b, int ib) {
  return a > b || (a == b && (unsigned)ia < (unsigned)ib);
}

// Work items of the batched IVF scan: (partition, chunk of <= qb of the
// (query, probe) pairs that probe it), partitions visited in `order`
// (largest first).  Pairs are sorted by partition; pair e belongs to query
// pair_vals[e] / tmax and writes its list to slot e.
struct IvfWork {
  const int64_t* part_off;
  const int64_t* pair_off;
  const int32_t* pair_vals;
  const int32_t* order;
  const int32_t* item_base;   // [c + 1], item_base[c] = total
  int c, tmax, qb;
  __device__ int count() const { return item_base[c]; }
  __device__ int partition_of(int item) const {
    int lo = 0, hi = c - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (item_base[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;   // index into `order`
  }
  __device__ void describe(int item, int64_t& r0, int64_t& r1, int64_t& e0, int& nqi) const {
    const int lo = partition_of(item);
    const int p = order[lo];
    e0 = pair_off[p] + (int64_t)(item - item_base[lo]) * qb;
    nqi = (int)min((int64_t)qb, pair_off[p + 1] - e0);
    r0 = part_off[p];
    r1 = part_off[p + 1];
  }
  __device__ int64_t query(int64_t e) const { return pair_vals[e] / tmax; }
  __device__ int64_t slot(int64_t e) const { return e; }
};

// Largest k of the tensor-core scan (its heap mode) and the largest
// candidate list per pair slot in that mode.
constexpr int kTcWideK = 128;
constexpr int kTcWideList = 256;

// Finishing of the tensor-core scan (finish_tc.cu), on the scan's candidate
// lists [nq * t][kc] and headers [nq * t] (L_k, count | overflow << 31):
// for k <= 32 the exact top k of every query into ids_out / scores_out;
// for k <= 128 every pair slot's list rescored exactly in place (best
// first, an id of -1 closing a shorter list) for the caller's merge.
void finish_tc_queries(const IndexData& ix, const Cand* lists, const int2* hdr, const int32_t* inv, int64_t nq,
                       int t, const int32_t* tpq, const float* Qf, const int32_t* top, int k, int kc,
                       int64_t* ids_out, float* scores_out, cudaStream_t s);
void rescore_tc_wide(const IndexData& ix, Cand* lists, const int2* hdr, const int32_t* inv,
                     const int32_t* pair_vals, int64_t nq, int t, const int32_t* tpq, const float* Qf,
                     const int32_t* top, int k, int kc, cudaStream_t s, Scratch& scr);

// Tensor-core scan (scan_tc.cu) of a fp32 index (rows in the core-matrix
// layout of tc.cuh, queries as fp32 rows of tc_kp columns): screening on the
// tensor cores, then exact rescoring.  For k <= 32 it also merges: the
// final top k of every query goes to ids_out / scores_out and it returns
// true.  Otherwise it leaves in `lists` one list of scan_tc_list_len(k)
// (exact score, id) entries per pair slot, best first, an id of -1 closing
// a shorter list, for the caller's merge, and returns false.
// k <= scan_tc_max_k(ix) (at most 128).
bool scan_tc_search(const IndexData& ix, const IvfWork& work, int max_items, const float* Qf, const float* qnorm,
                    const int32_t* top, const int32_t* inv, const int32_t* tpq, int64_t nq, int t, int k,
                    Cand* lists, int* err, int64_t* ids_out, float* scores_out, cudaStream_t s, Scratch& scr);
int scan_tc_max_k(const IndexData& ix);
// Candidate-list length per pair slot of the group-maxima scan (scan_gm.cu),
// which takes k <= 16 when its shared memory fits the row width.
constexpr int kGmList = 128;
bool scan_gm_usable(const IndexData& ix, int k);
// Launches it (after the caller cleared the headers, set the bounds to -inf
// and zeroed the work counter); lists [pairs][kGmList].
void scan_gm_launch(const IndexData& ix, const IvfWork& work, int grid, const float* Qf, const float* qnorm,
                    int64_t nq, int k, float dscale, long long wait_limit, int* counter, int* err,
                    unsigned* gbound, Cand* lists, int2* hdr, cudaStream_t s, Scratch& scr);
// SM cycles a pipeline wait of the scan may take before its CTA gives up
// (0: the default of about a second); the teardown's waits keep the default.
void set_scan_wait_limit(long long cycles);
int scan_tc_list_len(int k);

// Query-major exact scan (scan_query.cu): a warp per (query, probe) pair
// (top [nq][t], tpq per-query counts or null) over the core-matrix rows;
// lists [nq * t][k] get each pair's exact top k (k <= 32), best first, an id
// of -1 closing a shorter list, for the caller's k-way merge.  Usable when
// the batch probes few pairs per partition (nq * t <= 2c), k <= 32 and the
// rows have at most 1 024 columns.
bool scan_by_query_usable(const IndexData& ix, int64_t nq, int t, int k);
void scan_by_query(const IndexData& ix, const float* Qf, int qstride, const int32_t* top, const int32_t* tpq,
                   int64_t nq, int t, int k, Cand* lists, cudaStream_t s);

// FP8 shortlist (shortlist.cu): for every query the ids of the R best
// approximate scores s_q * s_x * sum q8 x8 over its probed union, each point
// once (its copy in the earliest-probed partition), padded with -1; Qf are
// the queries' code values (code_stride columns), qscale their scales.
void fp8_shortlist(const IndexData& ix, const float* Qf, const float* qscale, const int32_t* top,
                   const int32_t* tpq, int64_t nq, int t, int R, int32_t* cand, cudaStream_t s, Scratch& scr);
// The same shortlist for a PQ4 index: approximate score <q, C_p> + sum_s
// <q_s, B[s][code_s]> of each point's earliest-probed copy; Qf fp32 rows of
// qstride columns.
void pq_shortlist(const IndexData& ix, const float* Qf, int qstride, const int32_t* top, const int32_t* tpq,
                  int64_t nq, int t, int R, int32_t* cand, cudaStream_t s, Scratch& scr);

}  // namespace soar
