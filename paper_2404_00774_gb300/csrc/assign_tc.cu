// Primary and first spilled assignment on the 5th-generation tensor cores.
//
// One persistent CTA per SM takes tiles of 128 points.  The tile's points
// (and, for the spill, their unit residuals r_hat = (x - C[pi(x)]) / ||x - C[pi(x)]||)
// form the A operands in shared memory (fp32 rows in the K-major core-matrix
// layout of tc.cuh, staged by cp.async); the codebook, packed once per pass
// in that layout as B tiles of N = 256 centroids (128 for the spill) split
// into 8-column K steps, streams through a deep shared-memory ring of those
// K steps, copied by cp.async.bulk (it stays in L2: every CTA reads all of
// it, each CTA starting at its own tile).  Per K step one thread issues the
// kind::tf32 MMA X.C^T (and R.C^T for the spill) into a double-buffered TMEM
// accumulator; a wide N keeps the MMAs compute-bound rather than bound by
// re-reading the A tile from shared memory.  Eight epilogue warps read the
// scores back, one point per TMEM lane and half of the tile's columns per
// warp, and evaluate the expanded loss of Theorem 3.1
//     L(c') = ||c'||^2 - 2<x, c'> + lambda (<x, r_hat> - <c', r_hat>)^2
// (||x||^2 dropped: constant per point; lambda term absent for the primary).
//
// Rigorous screening.  kind::tf32 truncates each operand to 10 mantissa bits,
// so |<a, b>~ - <a, b>| < 2^-9 ||a|| ||b|| (fp32 accumulation is far below
// that).  With a factor-2 margin the screened loss of a pair is within
//     delta = 2^-7 ||x|| ||c'|| + lambda e (2 |t~| + e),  e = 2^-8 ||c'||,
// (t~ = <x, r_hat> - <c', r_hat>~) plus a small fp32 rounding allowance of the
// exact loss.  Per point the epilogue keeps the kList smallest lower bounds
// L~ - delta and the smallest upper bound U = min(L~ + delta); the true
// minimiser has lower bound <= U, so it is among the kept candidates unless
// more than kList lower bounds reach U (the point is then flagged and its
// refine pass scores every centroid).  Centroids the point is already
// assigned to are excluded (the spill reading of Section 3.3).  The refine
// kernel decides among the candidates with the direct form
// ||x - c'||^2 + lambda <x - c', r_hat>^2, lower index on ties.
//
// Warp roles: 0 = bulk-copy producer, 1 = TMEM owner and MMA issuer,
// 2..5 = epilogue and A-operand loaders.  Every mbarrier wait is bounded;
// on expiry the CTA raises *err, stops, waits (bounded) for its copies and
// MMAs in flight, frees its TMEM and returns.
#include <type_traits>

#include "internal.cuh"
#include "tc.cuh"

namespace soar {

namespace {

constexpr int kTM = 128;       // points per tile (MMA M)
constexpr int kEpi = 256;      // epilogue threads (8 warps: 4 lane quarters x 2 column halves)
constexpr int kThr = 96 + kEpi;   // producer, MMA issuer, gate, epilogue
constexpr int kStagesMax = 8;
constexpr int kStageBytes = 32768;   // codebook stage: 32 KB keeps bulk copies near full L2 bandwidth
constexpr int kList = 16;      // candidates kept per point
// parking area: a tile's 16 screened bounds per epilogue thread, overlaid at
// the end by the merge area (two lists of kList plus two scalars per point)
constexpr int kPark = 16 * kEpi > 2 * kList * kTM + 2 * kTM ? 16 * kEpi : 2 * kList * kTM + 2 * kTM;

// B tile width per pass: both fill the 512 TMEM columns with two buffers.
__host__ __device__ constexpr int tile_n(int ndir) { return ndir ? 128 : 256; }

template <typename XT>
struct AsgParams {
  const XT* X;
  int64_t n;
  int d, kp;
  const float* Cc;        // [ctiles][kp / 8][N][8] packed codebook (padding rows: zeros, +inf norm)
  const float* tmax;      // [ctiles] largest ||c|| of each B tile
  const float* C;         // [c][d] row-major
  int c, ctiles;
  int32_t* assign;        // [n][astride]: column 0 = primary (read by the spill pass); decided points written
  int astride;
  const float* inv_rn;    // [n][4] 1 / ||x - C[pi(x)]|| (0 for a zero residual)
  float lambda;
  int stages;
  int* counter;
  int* err;
  int32_t* cand;          // [n][kList] candidate centroids, -1 padded
  int32_t* ovf;           // [n] 1 when the candidates are not conclusive
  int32_t* queue;         // [n] points left to the refine
  int* qcount;
  int vec;                // fp32 rows, d % 4 == 0, X and C 16-byte aligned: 16-byte copies
};

__device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }

template <int NDIR, typename XT>
__global__ void __launch_bounds__(kThr, 1) assign_tc_kernel(AsgParams<XT> P) {
  constexpr int N = tile_n(NDIR);
  constexpr uint32_t kW = (1 + NDIR) * N;       // TMEM columns per accumulator buffer
  constexpr int kHalf = N / 2;                  // columns per epilogue thread and tile
  constexpr int G = kStageBytes / (N * 32);     // K steps per codebook stage
  // the no-swizzle operand layout needs 16-byte alignment only
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int kp = P.kp, S = P.stages, ksteps = kp / 8;
  const int nch = (ksteps + G - 1) / G;         // stages per B tile
  const uint32_t sbo = (uint32_t)kp * 32u;
  const uint32_t a_bytes = (uint32_t)kTM * kp * 4u;
  float* sX = reinterpret_cast<float*>(base);
  float* sR = reinterpret_cast<float*>(base + a_bytes);                       // spill only
  unsigned char* sB = base + (1 + NDIR) * (size_t)a_bytes;
  float* lb_s = reinterpret_cast<float*>(sB + (size_t)S * kStageBytes);      // [16][kEpi] parked bounds
  // merge area, overlaid on the parking area once every tile is done
  float* mlb_s = lb_s;                                                       // [kList][kTM]
  int* mid_s = reinterpret_cast<int*>(mlb_s + kList * kTM);                 // [kList][kTM]
  float* mu_s = reinterpret_cast<float*>(mid_s + kList * kTM);              // [kTM] U of the second half
  float* mev_s = mu_s + kTM;                                                // [kTM]
  float* nx_s = lb_s + kPark;                                               // [kTM] ||x||
  float* xr_s = nx_s + kTM;                                                 // [kTM] <x, r_hat>
  float* rn_s = xr_s + kTM;                                                 // [kTM] 1 or 0 (zero residual)
  int* prior_s = reinterpret_cast<int*>(rn_s + kTM);                        // [kTM]
  uint64_t* bars = reinterpret_cast<uint64_t*>(prior_s + kTM);
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s, issued_s, consumed_s, committed_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int s) { return tc::smem_u32(&bars[s]); };
  auto empty = [&](int s) { return tc::smem_u32(&bars[S + s]); };
  auto tfull = [&](int b) { return tc::smem_u32(&bars[2 * S + b]); };
  auto tempty = [&](int b) { return tc::smem_u32(&bars[2 * S + 2 + b]); };
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::bar_init(full(s), 1);
      tc::bar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::bar_init(tfull(b), 1);
      tc::bar_init(tempty(b), kEpi / 32);
    }
    tc::bar_init_fence();
    abort_s = 0;
    issued_s = consumed_s = committed_s = 0;
  }
  if (warp == 1) tc::tmem_alloc(tc::smem_u32(&tmem_base_s), 2 * kW);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base_s;
  const uint32_t idesc = tc::idesc_tf32(kTM, N);
  volatile int* abort_v = &abort_s;
  auto give_up = [&]() {
    if (atomicExch(&abort_s, 1) == 0) atomicExch(P.err, 1);
  };
  // epilogue thread: TMEM lane quarter q = warp % 4 (point row m), column half hh
  const int m = 32 * (warp & 3) + lane;
  const int hh = (warp - 3) >> 2;
  const int et = threadIdx.x - 96;              // epilogue thread index (parking column)

  // static schedule: items blockIdx.x, blockIdx.x + gridDim.x, ... so that the
  // producer can stream the codebook across item boundaries
  const int ntiles_pts = (int)((P.n + kTM - 1) / kTM);
  const int nitems = ntiles_pts > (int)blockIdx.x ? (ntiles_pts - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  // each CTA sweeps the codebook from its own starting tile, so that the SMs
  // do not all read the same L2 lines at the same moment
  const int rot = (int)(((int64_t)blockIdx.x * P.ctiles) / gridDim.x);

  if (warp == 0) {
    // ---- producer: the codebook stages of every item, back to back
    if (lane == 0) {
      uint32_t C = 0;
      bool stop = false;
      for (int it = 0; it < nitems && !stop; ++it)
        for (int i = 0; i < P.ctiles && !stop; ++i) {
          const int ti = (i + rot) % P.ctiles;
          for (int g = 0; g < nch; ++g, ++C) {
            const uint32_t s = C % S, ph = (C / S) & 1;
            if (!tc::bar_wait(empty(s), ph ^ 1, abort_v)) { give_up(); stop = true; break; }
            const int k0 = g * G, kn = min(G, ksteps - k0);
            const uint32_t bytes = (uint32_t)kn * N * 32;
            tc::bar_arrive_expect_tx(full(s), bytes);
            tc::bulk_copy_g2s(tc::smem_u32(sB) + s * kStageBytes, P.Cc + ((int64_t)ti * ksteps + k0) * N * 8,
                              bytes, full(s));
            issued_s = (int)(C + 1);
          }
        }
    }
  } else {
    uint32_t tile_ctr = 0, chunk_ctr = 0;
    uint32_t committed = 0;                     // MMA issuer: tiles whose tfull commit was issued
    for (int it = 0; it < nitems; ++it) {
      if (tc::named_bar_or(3, kThr - 32, *abort_v != 0)) break;   // (also ends the previous item)
      const int item = (int)blockIdx.x + it * (int)gridDim.x;
      const int64_t p = (int64_t)item * kTM + m;
      const bool active = warp >= 3 && p < P.n;

      // ---- A operands (first-half epilogue warps): the tile's points and
      // unit residuals, each row closed by (-1/2, -1/2) in columns d, d+1
      // against the codebook's (hi, lo) split of ||c||^2
      if (warp >= 3 && hh == 0) {
        float* xrow = sX + (m >> 3) * (kp * 8) + (m & 7) * 4;
        float* rrow = sR + (m >> 3) * (kp * 8) + (m & 7) * 4;
        float inv = 0.f;
        int prior = -1;
        const float* cr = nullptr;
        if (NDIR > 0 && active) {
          prior = P.assign[p * P.astride];
          inv = P.inv_rn[p * 4];
          cr = P.C + (int64_t)prior * P.d;
        }
        float ss = 0.f, xd = 0.f;
        const bool vec = std::is_same<XT, float>::value && P.vec;
        const int d4 = vec ? P.d / 4 : 0;               // 16-byte chunks staged by cp.async
        if (vec && active) {
          const float* xsrc = reinterpret_cast<const float*>(P.X) + p * P.d;
          for (int k4 = 0; k4 < d4; ++k4) tc::cp_async16(tc::smem_u32(xrow + k4 * 32), xsrc + 4 * k4);
          if (NDIR > 0)
            for (int k4 = 0; k4 < d4; ++k4) tc::cp_async16(tc::smem_u32(rrow + k4 * 32), cr + 4 * k4);
        }
        tc::cp_async_wait_all();
        for (int k4 = 0; k4 < kp / 4; ++k4) {
          float xv[4], rv[4], cv[4] = {0.f, 0.f, 0.f, 0.f};
          if (k4 < d4) {
            if (active) {
              const float4 a = *reinterpret_cast<const float4*>(xrow + k4 * 32);
              xv[0] = a.x; xv[1] = a.y; xv[2] = a.z; xv[3] = a.w;
              if (NDIR > 0) {
                const float4 b = *reinterpret_cast<const float4*>(rrow + k4 * 32);
                cv[0] = b.x; cv[1] = b.y; cv[2] = b.z; cv[3] = b.w;
              }
            } else {
              xv[0] = xv[1] = xv[2] = xv[3] = 0.f;
            }
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int k = 4 * k4 + u;
              xv[u] = (active && k < P.d) ? ld(P.X + p * P.d + k) : 0.f;
              if (NDIR > 0) cv[u] = (active && k < P.d) ? __ldg(cr + k) : 0.f;
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            ss = fmaf(xv[u], xv[u], ss);
            if (NDIR > 0) {
              rv[u] = (xv[u] - cv[u]) * inv;
              xd = fmaf(xv[u], rv[u], xd);
            }
            const int k = 4 * k4 + u;
            if (k == P.d || k == P.d + 1) xv[u] = -0.5f;
          }
          *reinterpret_cast<float4*>(xrow + k4 * 32) = make_float4(xv[0], xv[1], xv[2], xv[3]);
          if (NDIR > 0) *reinterpret_cast<float4*>(rrow + k4 * 32) = make_float4(rv[0], rv[1], rv[2], rv[3]);
        }
        nx_s[m] = sqrtf(ss);
        xr_s[m] = xd;                                  // <x, r_hat> of the stored (fp32) r_hat
        rn_s[m] = inv > 0.f ? 1.f : 0.f;
        prior_s[m] = prior;
        tc::fence_async_smem();
      }
      asm volatile("bar.sync 3, %0;" ::"n"(kThr - 32) : "memory");

      if (warp == 1) {
        // ---- MMA issuer.  It never touches an mbarrier (an mbarrier access
        // right after tcgen05.mma stalls the thread until the MMA pipe
        // drains): the gate warp waits for it and hands each codebook stage
        // over through a named barrier that also carries the stop flag.
        bool stop = false;
        for (int i = 0; i < P.ctiles && !stop; ++i) {
          const uint32_t T = tile_ctr + i, b = T & 1;
          for (int g = 0; g < nch; ++g) {
            stop = tc::named_bar_or(2, 64, false);
            if (stop) break;
            if (lane == 0) {
              const uint32_t C = chunk_ctr + i * nch + g, s = C % S;
              tc::fence_after_sync();
              const int k0 = g * G, kn = min(G, ksteps - k0);
              for (int jj = 0; jj < kn; ++jj) {
                const int j = k0 + jj;
                const uint64_t bd = tc::smem_desc(tc::smem_u32(sB) + s * kStageBytes + jj * N * 32, 128, 256);
                tc::mma_tf32(tmem + b * kW, tc::smem_desc(tc::smem_u32(sX) + j * 256, 128, sbo), bd, idesc, j > 0);
                if (NDIR > 0)
                  tc::mma_tf32(tmem + b * kW + N, tc::smem_desc(tc::smem_u32(sR) + j * 256, 128, sbo), bd, idesc,
                               j > 0);
              }
              tc::mma_commit(empty(s));              // the stage is free once these MMAs completed
            }
            __syncwarp();
          }
          if (lane == 0) tc::mma_commit(tfull(b));   // (also after a stop: MMAs in flight land first)
          committed = T + 1;
        }
        if (lane == 0) committed_s = (int)committed;
      } else if (warp == 2) {
        // ---- gate: waits for the TMEM buffer and each codebook stage, then
        // releases the MMA issuer
        bool stop = false;
        for (int i = 0; i < P.ctiles && !stop; ++i) {
          const uint32_t T = tile_ctr + i, b = T & 1, tph = (T >> 1) & 1;
          for (int g = 0; g < nch; ++g) {
            const uint32_t C = chunk_ctr + i * nch + g, s = C % S, ph = (C / S) & 1;
            int ok = 1;
            if (lane == 0) {
              ok = (g > 0 || tc::bar_wait(tempty(b), tph ^ 1, abort_v)) && tc::bar_wait(full(s), ph, abort_v);
              if (!ok) give_up();
              else consumed_s = (int)(C + 1);
              tc::fence_before_sync();
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            stop = tc::named_bar_or(2, 64, !ok);
            if (stop) break;
          }
        }
      } else {
        // ---- epilogue: kHalf of each B tile's N columns per thread
        float lbs[kList];
        int ids[kList];
#pragma unroll
        for (int j = 0; j < kList; ++j) { lbs[j] = INFINITY; ids[j] = -1; }
        float U = INFINITY, ev = INFINITY;
        const float nx = nx_s[m], xr = xr_s[m], er0 = ldexpf(rn_s[m], -8);
        const int prior = prior_s[m];
        const float lam = P.lambda;
        for (int i = 0; i < P.ctiles; ++i) {
          const uint32_t T = tile_ctr + i, b = T & 1, tph = (T >> 1) & 1;
          const bool ok = tc::bar_wait(tfull(b), tph, abort_v);
          if (!ok) give_up();
          tc::fence_after_sync();
          // per-tile bound: |L~ - L| <= dlc + 2 lambda e |t~| for every column
          const int ti = (i + rot) % P.ctiles;
          const float cmax = __ldg(P.tmax + ti), c2max = cmax * cmax;
          const float e = er0 * cmax;
          float dlc = fmaf(ldexpf(nx, -7), cmax, ldexpf(fmaf(nx, cmax, c2max), -14));
          if (NDIR > 0) dlc = fmaf(lam * e, e, fmaf(ldexpf(lam, -14), (nx + cmax) * (nx + cmax), dlc));
          const float two_le = 2.f * lam * e;
#pragma unroll 1
          for (int rd = 0; rd < kHalf / 32 && ok; ++rd) {
            const int col0 = hh * kHalf + 32 * rd;
            uint32_t rx[32], rr[32];
            const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + b * kW + col0;
            tc::tmem_ld32(taddr, rx);
            if (NDIR > 0) tc::tmem_ld32(taddr + N, rr);
            tc::tmem_ld_wait();
            const int cbase = ti * N + col0;
            const int jskip = (NDIR > 0) ? prior - cbase : -1;       // the point's own centroid
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
              const float worst0 = lbs[kList - 1];
              uint32_t mask = 0;
              // four interleaved partial minima keep the dependency chains
              // short; padded centroid rows carry ||c||^2 = +inf, so their
              // loss is +inf and they drop out without a test
              float um[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
              float evp[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
#pragma unroll
              for (int j2 = 0; j2 < 16; ++j2) {
                const int j = 16 * h2 + j2;
                float L = -2.f * __uint_as_float(rx[j]);
                float lb, ub;
                if constexpr (NDIR > 0) {
                  const float t = xr - __uint_as_float(rr[j]);
                  L = fmaf(lam * t, t, L);
                  const float dl = fmaf(two_le, fabsf(t), dlc);
                  lb = j == jskip ? INFINITY : L - dl;
                  ub = j == jskip ? INFINITY : L + dl;
                } else {
                  lb = L - dlc;
                  ub = L;                                   // + dlc once per round
                }
                um[j2 & 3] = fminf(um[j2 & 3], ub);
                const bool in = lb < worst0;
                evp[j2 & 3] = in ? evp[j2 & 3] : fminf(evp[j2 & 3], lb);
                if (in) {
                  mask |= 1u << j2;
                  lb_s[j2 * kEpi + et] = lb;
                }
              }
              float umin = fminf(fminf(um[0], um[1]), fminf(um[2], um[3]));
              if constexpr (NDIR == 0) umin += dlc;
              ev = fminf(ev, fminf(fminf(evp[0], evp[1]), fminf(evp[2], evp[3])));
              U = fminf(U, umin);
              for (; mask; mask &= mask - 1) {
                const int j2 = __ffs(mask) - 1;
                float v = lb_s[j2 * kEpi + et];
                if (!(v < lbs[kList - 1])) {
                  ev = fminf(ev, v);
                  continue;
                }
                ev = fminf(ev, lbs[kList - 1]);
                int id = cbase + 16 * h2 + j2;
#pragma unroll
                for (int q = 0; q < kList; ++q) {
                  if (v < lbs[q]) {
                    const float tv = lbs[q];
                    const int tid2 = ids[q];
                    lbs[q] = v;
                    ids[q] = id;
                    v = tv;
                    id = tid2;
                  }
                }
              }
            }
          }
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) tc::bar_arrive(tempty(b));
          if (!ok) break;
        }
        // merge the two column halves of each point (the merge area overlays
        // the parking area: every epilogue thread must be past its tiles)
        asm volatile("bar.sync 1, %0;" ::"n"(kEpi) : "memory");
        if (hh == 1) {
#pragma unroll
          for (int q = 0; q < kList; ++q) {
            mlb_s[q * kTM + m] = lbs[q];
            mid_s[q * kTM + m] = ids[q];
          }
          mu_s[m] = U;
          mev_s[m] = ev;
        }
        asm volatile("bar.sync 1, %0;" ::"n"(kEpi) : "memory");
        if (hh == 0 && active && !abort_s) {
          U = fminf(U, mu_s[m]);
          ev = fminf(ev, mev_s[m]);
          for (int q2 = 0; q2 < kList; ++q2) {
            float v = mlb_s[q2 * kTM + m];
            int id = mid_s[q2 * kTM + m];
            if (!(v < lbs[kList - 1])) {
              ev = fminf(ev, v);
              continue;
            }
            ev = fminf(ev, lbs[kList - 1]);
#pragma unroll
            for (int q = 0; q < kList; ++q) {
              if (v < lbs[q] || (v == lbs[q] && id < ids[q])) {
                const float tv = lbs[q];
                const int ti2 = ids[q];
                lbs[q] = v;
                ids[q] = id;
                v = tv;
                id = ti2;
              }
            }
          }
          int ncand = 0;
#pragma unroll
          for (int q = 0; q < kList; ++q) ncand += lbs[q] <= U ? 1 : 0;
          const bool over = ev <= U;
          if (ncand == 1 && !over) {
            P.assign[p * P.astride + NDIR] = ids[0];   // the bounds leave one centroid: decided
          } else {
#pragma unroll
            for (int q = 0; q < kList; ++q) P.cand[p * kList + q] = lbs[q] <= U ? ids[q] : -1;
            P.ovf[p] = over ? 1 : 0;
          }
          // queue the undecided points for the direct-form refine (one atomic per warp)
          const unsigned am = __activemask();
          const unsigned need = __ballot_sync(am, ncand != 1 || over);
          const int leader = __ffs(am) - 1;
          int qbase = 0;
          if (lane == leader && need) qbase = atomicAdd(P.qcount, __popc(need));
          qbase = __shfl_sync(am, qbase, leader);
          if (need & (1u << lane)) P.queue[qbase + __popc(need & ((1u << lane) - 1))] = (int32_t)p;
        }
      }
      tile_ctr += P.ctiles;
      chunk_ctr += (uint32_t)P.ctiles * nch;
    }
  }

  __syncthreads();
  if (abort_s && threadIdx.x == 0) {
    volatile int never = 0;
    for (int C = consumed_s; C < issued_s; ++C) tc::bar_wait(full(C % S), (C / S) & 1, &never);
  }
  if (abort_s && threadIdx.x == 64 && committed_s > 0) {
    volatile int never = 0;
    const int T = committed_s - 1;
    tc::bar_wait(tfull(T & 1), (T >> 1) & 1, &never);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, 2 * kW);
}

__global__ void codebook_norms(const float* __restrict__ C, int c, int d, float* __restrict__ n2,
                               float* __restrict__ n1) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= c) return;
  float s = 0.f;
  for (int k = lane; k < d; k += 32) {
    const float v = C[(int64_t)w * d + k];
    s = fmaf(v, v, s);
  }
  s = warp_sum(s);
  if (lane == 0) {
    n2[w] = s;
    n1[w] = sqrtf(s);
  }
}

// Codebook as B tiles of N rows, each split into K steps of 8 columns stored
// contiguously in the core-matrix layout of tc.cuh (8-row groups 256 bytes
// apart): rows padded to ctiles * N and columns to kp with zeros, except
// columns d and d + 1 holding ||c||^2 split into its tf32 part and the
// remainder (the MMA then adds -||c||^2 / 2 to <x, c> at full fp32 accuracy);
// padding rows hold +inf there.
__global__ void pack_codebook(const float* __restrict__ C, const float* __restrict__ n2, int c, int d, int kp,
                              int N, int rows_pad, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows_pad * kp) return;
  const int r = (int)(i / kp), k = (int)(i % kp);
  float v = 0.f;
  if (r < c) {
    if (k < d) {
      v = C[(int64_t)r * d + k];
    } else if (k <= d + 1) {
      const float hi = __uint_as_float(__float_as_uint(n2[r]) & 0xffffe000u);   // tf32 truncation
      v = k == d ? hi : n2[r] - hi;
    }
  } else if (k == d) {
    v = INFINITY;           // padding rows: infinite loss for every point
  }
  const int ti = r / N, rr = r % N, j = k >> 3, kk = k & 7;
  out[((int64_t)ti * (kp / 8) + j) * N * 8 + (rr >> 3) * 64 + (kk >> 2) * 32 + (rr & 7) * 4 + (kk & 3)] = v;
}

// Largest ||c|| of each N-centroid tile (warp per tile).
__global__ void tile_max_norms(const float* __restrict__ n1, int c, int N, int ctiles, float* __restrict__ tmax) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= ctiles) return;
  float v = 0.f;
  for (int j = lane; j < N; j += 32) {
    const int r = w * N + j;
    if (r < c) v = fmaxf(v, n1[r]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) tmax[w] = v;
}

// Direct-form decision among the candidates of each queued point (warp per
// point, persistent over the queue): two lanes per listed candidate, or,
// for a point the screen flagged, the lanes split every centroid not yet
// assigned to it.  Lower index on equal losses.
template <typename XT>
__global__ void refine_list(const XT* __restrict__ X, int d, const float* __restrict__ C, int c,
                            int32_t* __restrict__ assign, int astride, int col, float lambda,
                            const int32_t* __restrict__ cand, const int32_t* __restrict__ ovf,
                            const int32_t* __restrict__ queue, const int* __restrict__ qcount) {
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int total = *qcount;
  for (int64_t qi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; qi < total; qi += nwarps) {
    const int64_t p = queue[qi];
    const XT* x = X + p * d;
    const int prior = col > 0 ? assign[p * astride] : -1;
    const float* cr = C + (int64_t)(col > 0 ? prior : 0) * d;
    float rn2 = 0.f;
    if (col > 0) {
      float s = 0.f;
      for (int k = lane; k < d; k += 32) {
        const float v = load_elem(x, k) - cr[k];
        s = fmaf(v, v, s);
      }
      rn2 = warp_sum(s);
    }
    float best = INFINITY;
    int bi = -1;
    const bool listed = !ovf[p] && cand[p * kList] >= 0;
    if (listed) {
      static_assert(kList * 2 == 32, "two lanes per candidate");
      const int g = lane >> 1, part = lane & 1;
      const int cq = cand[p * kList + g];
      float dist = 0.f, pr = 0.f;
      if (cq >= 0) {
        const float* cv = C + (int64_t)cq * d;
        for (int k = part; k < d; k += 2) {
          const float xv = load_elem(x, k);
          const float v = xv - cv[k];
          dist = fmaf(v, v, dist);
          if (col > 0) pr = fmaf(v, xv - cr[k], pr);
        }
      }
#pragma unroll
      for (int o = 1; o < 2; o <<= 1) {
        dist += __shfl_xor_sync(kFull, dist, o);
        pr += __shfl_xor_sync(kFull, pr, o);
      }
      if (cq >= 0) {
        best = (col > 0 && rn2 > 0.f) ? fmaf(lambda, pr * pr / rn2, dist) : dist;
        bi = cq;
      }
    } else {
      for (int cq = lane; cq < c; cq += 32) {
        if (cq == prior) continue;
        const float* cv = C + (int64_t)cq * d;
        float dist = 0.f, pr = 0.f;
        for (int k = 0; k < d; ++k) {
          const float xv = load_elem(x, k);
          const float v = xv - cv[k];
          dist = fmaf(v, v, dist);
          if (col > 0) pr = fmaf(v, xv - cr[k], pr);
        }
        const float l = (col > 0 && rn2 > 0.f) ? fmaf(lambda, pr * pr / rn2, dist) : dist;
        if (l < best || (l == best && (unsigned)cq < (unsigned)bi)) { best = l; bi = cq; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(kFull, best, o);
      const int oi = __shfl_xor_sync(kFull, bi, o);
      if (oi >= 0 && (bi < 0 || ob < best || (ob == best && oi < bi))) { best = ob; bi = oi; }
    }
    if (lane == 0) assign[p * astride + col] = bi;
  }
}

size_t smem_for(int kp, int ndir, int s) {
  return 128 + (size_t)(1 + ndir) * kTM * kp * 4 + (size_t)s * kStageBytes + (size_t)kPark * 4 +
         (size_t)4 * kTM * 4 + (size_t)(2 * s + 4) * 8;
}

// K of the MMAs: d columns plus the two norm columns, a multiple of 8
int kp_for(int d) { return (d + 2 + 7) / 8 * 8; }

int stages_for(int kp, int ndir) {
  for (int s = kStagesMax; s >= 2; --s)
    if (smem_for(kp, ndir, s) <= 227 * 1024 - 256) return s;   // room for the static shared variables
  return 0;
}

}  // namespace

bool assign_tc_supported(int d, int ndir) { return ndir <= 1 && stages_for(kp_for(d), ndir) >= 2; }

template <typename XT>
void assign_tc_pass(const XT* X, int64_t n, int d, const float* C, int c, int ndir, int32_t* assign, int astride,
                    const float* inv_rn, float lambda, cudaStream_t s, Scratch& scr) {
  const int kp = kp_for(d);
  const int stages = stages_for(kp, ndir);
  if (ndir > 1 || stages < 2) fail(SOAR_EUNSUPPORTED, "tensor-core assignment: unsupported shape");
  const int N = tile_n(ndir);
  const int ctiles = (c + N - 1) / N;
  float* Cc = scr.get<float>((size_t)ctiles * N * kp);
  float* n2 = scr.get<float>(c);
  float* n1 = scr.get<float>(c);
  float* tmax = scr.get<float>(ctiles);
  codebook_norms<<<ceil_div((int64_t)c * 32, 256), 256, 0, s>>>(C, c, d, n2, n1);
  SOAR_LAUNCHED();
  pack_codebook<<<ceil_div((int64_t)ctiles * N * kp, 256), 256, 0, s>>>(C, n2, c, d, kp, N, ctiles * N, Cc);
  SOAR_LAUNCHED();
  tile_max_norms<<<ceil_div((int64_t)ctiles * 32, 256), 256, 0, s>>>(n1, c, N, ctiles, tmax);
  SOAR_LAUNCHED();
  int32_t* cand = scr.get<int32_t>((size_t)n * kList);
  int32_t* ovf = scr.get<int32_t>(n);
  int32_t* queue = scr.get<int32_t>(n);
  int* counter = scr.get<int>(2);            // work items, queued points
  SOAR_CUDA(cudaMemsetAsync(counter, 0, 2 * sizeof(int), s));
  const int vec = std::is_same<XT, float>::value && d % 4 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0 &&
                  reinterpret_cast<uintptr_t>(C) % 16 == 0;
  AsgParams<XT> prm{X, n, d, kp, Cc, tmax, C, c, ctiles, assign, astride, inv_rn, lambda, stages,
                    counter, device_error_word(), cand, ovf, queue, counter + 1, vec};
  const size_t smem = smem_for(kp, ndir, stages);
  auto kern = ndir == 0 ? assign_tc_kernel<0, XT> : assign_tc_kernel<1, XT>;
  SOAR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = (int)std::min<int64_t>((n + kTM - 1) / kTM, num_sms());
  kern<<<grid, kThr, smem, s>>>(prm);
  SOAR_LAUNCHED();
  refine_list<XT><<<num_sms() * 8, 256, 0, s>>>(X, d, C, c, assign, astride, ndir, lambda, cand, ovf, queue,
                                                  counter + 1);
  SOAR_LAUNCHED();
}

template void assign_tc_pass<float>(const float*, int64_t, int, const float*, int, int, int32_t*, int, const float*,
                                    float, cudaStream_t, Scratch&);
template void assign_tc_pass<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int, const float*, int, int, int32_t*,
                                            int, const float*, float, cudaStream_t, Scratch&);

}  // namespace soar
