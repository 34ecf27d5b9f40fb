// Exact finishing of the tensor-core partition scan (scan_tc.cu): the
// screened candidate lists of every (query, partition) pair are rescored
// exactly in fp32 (fp32 rows, or bf16 rows widened exactly) from the
// row-major copy of the index, the partitions
// whose lists overflowed are rescanned exactly, spilled copies of a point
// are dropped (Section 3.5: a spilled point's copies carry bit-identical
// exact scores) and each query keeps its top k (Section 2.2).
//   k <= 32   finish_queries: a warp per query, rescoring and merge fused
//   k <= 128  query_bounds + rescore_wide: a warp per (query, partition)
//             slot, leaving one exact list per slot for the caller's merge
#include "scan_common.cuh"

namespace soar {

namespace {

constexpr int kWideK = kTcWideK;   // largest k of the heap mode
constexpr int kWideList = kTcWideList;   // largest candidate list per slot in that mode

// Largest L_k over each query's partitions: a lower bound of its final k-th
// best exact score.
__global__ void query_bounds(const int2* __restrict__ hdr, const int32_t* __restrict__ inv, int64_t nq, int t,
                             const int32_t* __restrict__ tpq, float* __restrict__ lstar) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int tq = tpq ? min(max(tpq[q], 0), t) : t;
  float best = -INFINITY;
  for (int j = 0; j < tq; ++j) best = fmaxf(best, __int_as_float(hdr[inv[q * t + j]].x));
  lstar[q] = best;
}

// Exact fp32 <q, x> of row-major row `pos` (row stride rs; k ascending, the
// same order for every copy of a point).  fp32 rows: rs a multiple of 4.
__device__ __forceinline__ float exact_dot_rm(const float* __restrict__ q, const float* __restrict__ vec, int rs,
                                              int64_t pos) {
  const float* x = vec + pos * (int64_t)rs;
  float acc = 0.f;
#pragma unroll 8
  for (int k4 = 0; k4 < rs / 4; ++k4) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(q + 4 * k4));
    const float4 v = __ldg(reinterpret_cast<const float4*>(x + 4 * k4));
    acc = fmaf(a.x, v.x, acc);
    acc = fmaf(a.y, v.y, acc);
    acc = fmaf(a.z, v.z, acc);
    acc = fmaf(a.w, v.w, acc);
  }
  return acc;
}

// bf16 rows (rs a multiple of 8): each element widened to fp32 exactly.
__device__ __forceinline__ float exact_dot_rm(const float* __restrict__ q, const __nv_bfloat16* __restrict__ vec,
                                              int rs, int64_t pos) {
  const __nv_bfloat16* x = vec + pos * (int64_t)rs;
  float acc = 0.f;
#pragma unroll 4
  for (int k8 = 0; k8 < rs / 8; ++k8) {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(x + 8 * k8));
    const float4 a0 = __ldg(reinterpret_cast<const float4*>(q + 8 * k8));
    const float4 a1 = __ldg(reinterpret_cast<const float4*>(q + 8 * k8 + 4));
    acc = fmaf(a0.x, __uint_as_float(w.x << 16), acc);
    acc = fmaf(a0.y, __uint_as_float(w.x & 0xffff0000u), acc);
    acc = fmaf(a0.z, __uint_as_float(w.y << 16), acc);
    acc = fmaf(a0.w, __uint_as_float(w.y & 0xffff0000u), acc);
    acc = fmaf(a1.x, __uint_as_float(w.z << 16), acc);
    acc = fmaf(a1.y, __uint_as_float(w.z & 0xffff0000u), acc);
    acc = fmaf(a1.z, __uint_as_float(w.w << 16), acc);
    acc = fmaf(a1.w, __uint_as_float(w.w & 0xffff0000u), acc);
  }
  return acc;
}


// Rescoring for 32 < k <= 128 (heap mode, lists of kc <= 256 entries), a
// warp per (query, partition) slot: the candidates whose upper bound reaches
// the query's bound are rescored exactly and the best k kept;
// a slot whose list overflowed is rescanned exactly over its partition into
// a shared-memory top-k list.  The slot is rewritten best first and closed
// by a (-inf, -1) entry when shorter than kc.
template <typename RowT>
__global__ void __launch_bounds__(256) rescore_wide(Cand* __restrict__ cand, const int2* __restrict__ hdr, int64_t P,
                                                    const int32_t* __restrict__ pair_vals, int t,
                                                    const float* __restrict__ lstar, const float* __restrict__ Qf,
                                                    int kp, const RowT* __restrict__ rows, int rs,
                                                    const int32_t* __restrict__ ids,
                                                    const int32_t* __restrict__ part_of_pair,
                                                    const int64_t* __restrict__ gstart,
                                                    const int64_t* __restrict__ part_off, int k, int kc,
                                                    const int32_t* __restrict__ tpq) {
  constexpr unsigned kFull = 0xffffffffu;
  constexpr int R = kWideList / 32;       // candidates per lane
  constexpr int U = kWideK / 32;          // top-k entries per lane
  __shared__ Cand top_s[8][kWideK];
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // uniform within a warp
  const int lane = threadIdx.x & 31;
  if (e >= P) return;
  const int64_t q = pair_vals[e] / t;
  const int j = pair_vals[e] - (int)(q * t);
  if (tpq && j >= min(max(tpq[q], 0), t)) return;
  const int2 h = hdr[e];
  const int cnt = min(h.y & 0x7fffffff, kc);
  const bool ovf = h.y < 0;
  const float bound = lstar[q];
  const float* qv = Qf + q * (int64_t)kp;
  Cand* slot = cand + e * (int64_t)kc;
  if (!ovf) {
    float v[R];
    int id[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int idx = lane + 32 * r;
      v[r] = -INFINITY;
      id[r] = -1;
      if (idx < cnt) {
        const Cand c = slot[idx];
        if (c.s >= bound) {
          v[r] = exact_dot_rm(qv, rows, rs, c.id);
          id[r] = ids[c.id];
        }
      }
    }
    __syncwarp();
    int out = 0;
    for (; out < k; ++out) {
      float bs = v[0];
      int bid = id[0], br = 0;
#pragma unroll
      for (int r = 1; r < R; ++r)
        if (better(v[r], id[r], bs, bid)) { bs = v[r]; bid = id[r]; br = r; }
      float ws = bs;
      int wid = bid, wl = lane;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float os = __shfl_xor_sync(kFull, ws, o);
        const int oid = __shfl_xor_sync(kFull, wid, o);
        const int ol = __shfl_xor_sync(kFull, wl, o);
        if (better(os, oid, ws, wid) || (os == ws && oid == wid && ol < wl)) { ws = os; wid = oid; wl = ol; }
      }
      if (wid == -1) break;                  // every candidate taken
      if (lane == wl) {
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r == br) { v[r] = -INFINITY; id[r] = -1; }
      }
      if (lane == 0) slot[out] = Cand{ws, wid};
    }
    if (lane == 0 && out < kc) slot[out] = Cand{-INFINITY, -1};
    return;
  }
  // overflow: exact rescan of the partition
  Cand* L = top_s[threadIdx.x >> 5];
  for (int i = lane; i < k; i += 32) L[i] = Cand{-INFINITY, -1};
  __syncwarp();
  const int p = part_of_pair[e];
  const int64_t r0 = part_off[p];
  const int64_t nrows = part_off[p + 1] - part_off[p];
  for (int64_t base = 0; base < nrows; base += 32) {
    const int64_t r = base + lane;
    float v = -INFINITY;
    int rid = -1;
    if (r < nrows) {
      v = exact_dot_rm(qv, rows, rs, r0 + r);
      rid = ids[r0 + r];
    }
    unsigned ball = __ballot_sync(kFull, r < nrows && better(v, rid, L[k - 1].s, L[k - 1].id));
    while (ball) {
      const int src = __ffs(ball) - 1;
      ball &= ball - 1;
      const float vs = __shfl_sync(kFull, v, src);
      const int is = __shfl_sync(kFull, rid, src);
      if (!better(vs, is, L[k - 1].s, L[k - 1].id)) continue;   // same answer in every lane
      int nb = 0;                                              // entries better than (vs, is)
      for (int i = lane; i < k; i += 32) nb += better(L[i].s, L[i].id, vs, is) ? 1 : 0;
      nb = __reduce_add_sync(kFull, nb);
      Cand tmp[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = lane + 32 * u;
        if (i >= nb && i < k - 1) tmp[u] = L[i];
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = lane + 32 * u;
        if (i >= nb && i < k - 1) L[i + 1] = tmp[u];
      }
      __syncwarp();
      if (lane == 0) L[nb] = Cand{vs, is};
      __syncwarp();
    }
  }
  for (int i = lane; i < k; i += 32) slot[i] = L[i];
  if (lane == 0 && k < kc) slot[k] = Cand{-INFINITY, -1};
}

// Finishing pass for k <= 32, a warp per query: the query's bound L* (the
// largest L_k of its partitions) bounds its final k-th best exact score from
// below; every candidate whose upper bound reaches L* (and beats the current
// k-th best) is rescored exactly, and every partition whose list overflowed
// is rescanned exactly.  The exact results go into a lane-distributed sorted
// top-k (lane j: j-th best rank key), dropping the second copy of a spilled
// point (its exact score is bit-identical, so its key is too).  Writes the
// query's ids / scores, padded with -1 / -inf.
template <typename RowT>
__global__ void __launch_bounds__(256) finish_queries(
    const Cand* __restrict__ cand, const int2* __restrict__ hdr, const int32_t* __restrict__ inv, int64_t nq, int t,
    const int32_t* __restrict__ tpq, const float* __restrict__ Qf, int kp, const RowT* __restrict__ rows, int rs,
    const int32_t* __restrict__ ids, const int32_t* __restrict__ top, const int64_t* __restrict__ gstart,
    const int64_t* __restrict__ part_off, int k, int kc, int64_t* __restrict__ ids_out,
    float* __restrict__ scores_out) {
  constexpr unsigned kFull = 0xffffffffu;
  constexpr int kPend = 256;                    // pending candidates per warp
  __shared__ int32_t pend_s[8][kPend];
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= nq) return;
  const int tq = tpq ? min(max(tpq[q], 0), t) : t;
  float lstar = -INFINITY;
  for (int j = lane; j < tq; j += 32) lstar = fmaxf(lstar, __int_as_float(hdr[inv[q * t + j]].x));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lstar = fmaxf(lstar, __shfl_xor_sync(kFull, lstar, o));
  const float* qv = Qf + q * (int64_t)kp;
  uint64_t mine = ~0ull;          // lane j < k: the j-th best key so far (empty: after every real key)
  uint64_t thr = ~0ull;           // the k-th best key
  // inserts the keys of this round (one per lane, ~0 for none)
  auto insert_round = [&](uint64_t key) {
    unsigned bal = __ballot_sync(kFull, key < thr);
    while (bal) {
      const int src = __ffs(bal) - 1;
      bal &= bal - 1;
      const uint64_t kk = __shfl_sync(kFull, key, src);
      if (kk >= thr) continue;                                   // the same in every lane
      if (__ballot_sync(kFull, lane < k && mine == kk)) continue;  // spilled copy already in
      const int pos = __popc(__ballot_sync(kFull, lane < k && mine < kk));
      const uint64_t up = __shfl_up_sync(kFull, mine, 1);
      if (lane > pos && lane < k) mine = up;
      if (lane == pos) mine = kk;
      thr = __shfl_sync(kFull, mine, k - 1);
    }
  };
  // candidates whose upper bound reaches L*, gathered over all of the
  // query's partitions (padded row positions), then rescored 32 at a time so
  // that the exact dot products of a round overlap
  int32_t* pend = pend_s[threadIdx.x >> 5];
  int npend = 0;
  auto flush = [&]() {
    for (int b = 0; b < npend; b += 32) {
      const float kth = thr == ~0ull ? -INFINITY : key_float(~(uint32_t)(thr >> 32));
      uint64_t key = ~0ull;
      if (b + lane < npend) {
        const int32_t pos = pend[b + lane];
        const float v = exact_dot_rm(qv, rows, rs, pos);
        if (v >= kth) key = rank_key(v, (uint32_t)ids[pos]);
      }
      insert_round(key);
    }
    npend = 0;
    __syncwarp();
  };
  // the query's probes 32 at a time: lane l holds probe j0 + l's slot and
  // list length; a warp prefix sum over the lengths lets every lane load one
  // candidate of any of the 32 lists in the same round
  for (int j0 = 0; j0 < tq; j0 += 32) {
    const int j = j0 + lane;
    int64_t e_l = 0;
    int cnt_l = 0;
    bool ovf_l = false;
    if (j < tq) {
      e_l = inv[q * t + j];
      const int hy = hdr[e_l].y;
      ovf_l = hy < 0;
      cnt_l = ovf_l ? 0 : min(hy & 0x7fffffff, kc);
    }
    int incl = cnt_l;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    for (int base = 0; base < total; base += 32) {
      const int f = base + lane;
      // the list holding entry f: the first lane whose inclusive sum exceeds f
      int lo = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int probe = __shfl_sync(kFull, incl, lo + step - 1);
        if (probe <= f) lo += step;
      }
      const int64_t e = __shfl_sync(kFull, e_l, lo);
      const int first = __shfl_sync(kFull, incl, lo) - __shfl_sync(kFull, cnt_l, lo);
      bool keep = false;
      int32_t pos = 0;
      if (f < total) {
        const Cand c = cand[e * kc + (f - first)];
        keep = c.s >= lstar;
        pos = c.id;
      }
      const unsigned kb = __ballot_sync(kFull, keep);
      if (npend + __popc(kb) > kPend) flush();
      if (keep) pend[npend + __popc(kb & ((1u << lane) - 1u))] = pos;
      npend += __popc(kb);
      __syncwarp();
    }
    // lists that overflowed: rescan their partitions exactly
    for (unsigned ob = __ballot_sync(kFull, ovf_l); ob; ob &= ob - 1) {
      const int l = __ffs(ob) - 1;
      flush();
      const int p = top[q * t + j0 + l];
      const int64_t r0 = part_off[p];
      const int64_t nrows = part_off[p + 1] - part_off[p];
      for (int64_t rb = 0; rb < nrows; rb += 32) {
        const int64_t r = rb + lane;
        const uint64_t key = r < nrows ? rank_key(exact_dot_rm(qv, rows, rs, r0 + r), (uint32_t)ids[r0 + r]) : ~0ull;
        insert_round(key);
      }
    }
  }
  flush();
  if (lane < k) {
    const bool have = mine != ~0ull;
    ids_out[q * k + lane] = have ? (int64_t)(uint32_t)(mine & 0xffffffffu) : -1;
    scores_out[q * k + lane] = have ? key_float(~(uint32_t)(mine >> 32)) : -INFINITY;
  }
}


// partition of every sorted pair (for the overflow rescans)
__global__ void pair_partitions(const int32_t* __restrict__ top, const int32_t* __restrict__ pair_vals, int64_t P,
                                int32_t* __restrict__ part) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < P) part[e] = top[pair_vals[e]];
}

}  // namespace

void finish_tc_queries(const IndexData& ix, const Cand* lists, const int2* hdr, const int32_t* inv, int64_t nq,
                       int t, const int32_t* tpq, const float* Qf, const int32_t* top, int k, int kc,
                       int64_t* ids_out, float* scores_out, cudaStream_t s) {
  if (ix.dtype == SOAR_F32)
    finish_queries<float><<<ceil_div(nq * 32, 256), 256, 0, s>>>(lists, hdr, inv, nq, t, tpq, Qf, ix.tc_kp,
                                                                 static_cast<const float*>(ix.vectors), ix.row_stride,
                                                                 ix.ids, top, ix.tc_gstart, ix.offsets, k, kc,
                                                                 ids_out, scores_out);
  else
    finish_queries<__nv_bfloat16><<<ceil_div(nq * 32, 256), 256, 0, s>>>(
        lists, hdr, inv, nq, t, tpq, Qf, ix.tc_kp, static_cast<const __nv_bfloat16*>(ix.vectors), ix.row_stride,
        ix.ids, top, ix.tc_gstart, ix.offsets, k, kc, ids_out, scores_out);
  SOAR_LAUNCHED();
}

void rescore_tc_wide(const IndexData& ix, Cand* lists, const int2* hdr, const int32_t* inv,
                     const int32_t* pair_vals, int64_t nq, int t, const int32_t* tpq, const float* Qf,
                     const int32_t* top, int k, int kc, cudaStream_t s, Scratch& scr) {
  const int64_t P = nq * t;
  float* lstar = scr.get<float>(nq);
  query_bounds<<<ceil_div(nq, 256), 256, 0, s>>>(hdr, inv, nq, t, tpq, lstar);
  SOAR_LAUNCHED();
  int32_t* part = scr.get<int32_t>(P);
  pair_partitions<<<ceil_div(P, 256), 256, 0, s>>>(top, pair_vals, P, part);
  SOAR_LAUNCHED();
  if (ix.dtype == SOAR_F32)
    rescore_wide<float><<<ceil_div(P * 32, 256), 256, 0, s>>>(lists, hdr, P, pair_vals, t, lstar, Qf, ix.tc_kp,
                                                              static_cast<const float*>(ix.vectors), ix.row_stride,
                                                              ix.ids, part, ix.tc_gstart, ix.offsets, k, kc, tpq);
  else
    rescore_wide<__nv_bfloat16><<<ceil_div(P * 32, 256), 256, 0, s>>>(
        lists, hdr, P, pair_vals, t, lstar, Qf, ix.tc_kp, static_cast<const __nv_bfloat16*>(ix.vectors),
        ix.row_stride, ix.ids, part, ix.tc_gstart, ix.offsets, k, kc, tpq);
  SOAR_LAUNCHED();
}

}  // namespace soar
