// sdf.cu -- sm_103a kernels and host orchestration behind include/sdf.h.
//
// Method (paper sections / equations / algorithms):
//   S = mass I + w A^T A                      Sec. 2.1.2 Eq. schur (w = alpha kscale^2/mass)
//   primal active-set loop                    App. B.1 Algorithm pdas
//   restricted system, b = rhs_I - S_IA psi_A Sec. 2.1.2 Eq. reduced
//   A-DEF2 deflated Jacobi-PCG                Sec. 2.2.1 Algorithm adef2 (standard
//                                             Tang/Gaul form: p = P D^-1 r + beta p)
//   Z = orth(Phi|_I), E = Z^T S_II Z, guard   Sec. 2.2.2, Alg. online_deflation l. 5-15
//   stop on ||r|| <= rtol ||b||               App. B.2 Eq. cg_stop
//
// B300 design (what differs from the paper's CSR/cuSPARSE implementation):
//   * S is never assembled.  S_II u is applied matrix-free in flux form on
//     shared-memory tiles with a 2-node halo: w = A u on the halo ring, then
//     mass u + w A^T w on the tile, masked by the active-set bytes (vectors live
//     in full-grid layout with zeros on A, so no compaction).
//   * Only the shared reference modes Phi are read in the loop (no per-instance
//     N x k arrays): P z = z - Phi_I E_raw^-1 Phi_I^T S_II z, where
//     E_raw = Phi_I^T S_II Phi_I.  This equals Z E^-1 Z^T S_II for
//     Z = Phi_I R^-1 (Cholesky-QR, G = Phi_I^T Phi_I = R^T R); cond(E) for the
//     guard uses the orthonormal-basis E = R^-T E_raw R^-1.
//   * The k x k coarse operator is applied as an explicit GEMV with
//     E_raw^-1 = (L_e^-1 L_g^-1)^T (L_e^-1 L_g^-1), computed once per outer
//     iteration, instead of two sequential triangular solves per iteration.
//   * Reductions are deterministic: per-block partials, summed in block order
//     by the last block to finish (atomic ticket), no floating-point atomics.
//   * CG runs as three kernels per iteration; per-instance convergence flags
//     make finished instances' blocks exit at once, so the host enqueues
//     `check_every` iterations between polls.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <map>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "sdf_device.cuh"
#include "tc_device.cuh"
#include "host_linalg.h"

using namespace sdf;

namespace {

// Per-instance solver state (device, in the workspace).
struct InstState {
  double rho, sigma, alpha, beta, gamma, csign;
  double rnorm2, bnorm2;
  double rho_prev;     // rho before the last CG iteration (correction-pass beta)
  double floor2;       // mixed path: (floor_c u || |S_II||x| ||)^2 when last evaluated, else 0
  double rt2_prev;     // mixed path: true ||r||^2 at the previous residual replacement
  int32_t phase;       // 1: the coarse-correction pass is the next K_B/K_C
  int32_t cg_done;     // current inner solve finished (or failed)
  int32_t outer_done;  // instance finished
  int32_t iters;       // CG iterations of the current inner solve
  int32_t deflate;     // A-DEF2 in force for the current inner solve
  int32_t outer;       // index of the current inner solve
  int32_t changes;     // active-set changes of the last update
  int32_t empty_I;     // every node active: nothing to solve
  int32_t await;       // mixed path: recurrence residual met rtol, waiting for the FP64 check
  int32_t stall;       // mixed path: the true residual stalled at the last replacement
  double t[SDF_MAX_K]; // reduced projection Phi_I^T v
  sdf_stats stats;
};

enum { CNT_SETUP = 0, CNT_SIGMA = 1, CNT_UPDATE = 2, CNT_PROJECT = 3, CNT_ACTIVE = 4, NCNT = 5 };

struct Ctrl {       // grid-wide control words (device)
  int running;      // instances still iterating in the current inner solve
  int live;         // instances that need another outer iteration
  int pad[62];
};

struct Layout {
  size_t x, b64, r, r2, p, q, w, dinv, mask, W, Einv, Eraw, G, coarse, part, gpart, state, cnt,
      ctrl, v, cvec, ppart, xlo, total;
  int gx, gxa, gxg, gxp, nb, bpad, gxc, zc;
  int tcp, nbp;  // tensor-core projection (BF16 modes, batch <= 256) and its padded batch
  int tce, kp;   // tensor-core expansion and the padded mode count of its node-major copy
  size_t phin;   // node-major BF16 copy of the modes (tensor-core expansion)
  int fb;        // FP64 path with the shared-Phi batch kernels (batch >= kFp64BatchMin)
  int pairs;     // mixed 3D path: stencil kernels on instance pairs (packed FP32)
};

inline size_t al(size_t v) { return (v + 255) & ~size_t(255); }

// dynamic shared memory of k_expand_tc: the mode tile (128 nodes x KP) and
// three BF16 terms of the coefficients (NBP x KP), in 64-wide K blocks
inline size_t expand_tc_smem(int nbp, int kp) {
  const size_t nkb = (kp + 63) / 64;
  return nkb * 128 * 64 * 2 + 3 * nkb * (size_t)nbp * 64 * 2;
}

// ---------------------------------------------------------------------------
// helpers

// Upwind coefficients b_d / h_d of an instance; on a space-time problem the
// time axis takes 1 / dt instead (implicit Euler, App. E.2), whatever b_z is.
__device__ __forceinline__ void inst_cb(const OpParams &P, const double *inst, double cb[3]) {
  for (int d = 0; d < 3; ++d) cb[d] = (P.inst_conv && d < P.dim) ? inst[4 + d] * P.inv_h[d] : 0.0;
  if (P.time_axis) cb[2] = P.cb_t;
}

__device__ __forceinline__ double desired(const OpParams &P, const double *inst, int gx, int gy,
                                          int gz) {
  double dx = (gx + 1) * P.h[0] - inst[1];
  double dy = (gy + 1) * P.h[1] - inst[2];
  double r2 = dx * dx + dy * dy;
  if (P.time_axis) {  // App. F.5: the spatial Gaussian ramped in time
    const double t = (gz + 1) * P.dt;
    return (1.0 - exp(-t / P.ramp_tau)) * inst[0] * exp(-r2 / (2.0 * P.yd_sigma * P.yd_sigma));
  }
  if (P.dim == 3) {
    double dz = (gz + 1) * P.h[2] - inst[3];
    r2 += dz * dz;
  }
  return inst[0] * exp(-r2 / (2.0 * P.yd_sigma * P.yd_sigma));
}

// ---------------------------------------------------------------------------
// problem set-up: face coefficients and the shared Jacobi diagonal

__global__ void k_faces(OpParams P, const double *kappa, double diff_scale, double *fx,
                        double *fy, double *fz, float *fxf, float *fyf, float *fzf) {
  long long nfx = (long long)(P.nx + 1) * P.ny * P.nz;
  long long nfy = (long long)P.nx * (P.ny + 1) * P.nz;
  long long nfz = P.dim == 3 ? (long long)P.nx * P.ny * (P.nz + 1) : 0;
  auto kap = [&](int i, int j, int l) { return kappa[i + (long long)P.nx * (j + (long long)P.ny * l)]; };
  auto hm = [](double a, double b) { return 2.0 * a * b / (a + b); };
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nfx + nfy + nfz;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < nfx) {
      int i = (int)(e % (P.nx + 1));
      long long t = e / (P.nx + 1);
      int j = (int)(t % P.ny), l = (int)(t / P.ny);
      double kf = i == 0 ? kap(0, j, l) : i == P.nx ? kap(P.nx - 1, j, l) : hm(kap(i - 1, j, l), kap(i, j, l));
      fx[e] = diff_scale * kf * P.inv_h[0] * P.inv_h[0];
      fxf[e] = (float)fx[e];
    } else if (e < nfx + nfy) {
      long long f = e - nfx;
      int i = (int)(f % P.nx);
      long long t = f / P.nx;
      int j = (int)(t % (P.ny + 1)), l = (int)(t / (P.ny + 1));
      double kf = j == 0 ? kap(i, 0, l) : j == P.ny ? kap(i, P.ny - 1, l) : hm(kap(i, j - 1, l), kap(i, j, l));
      fy[f] = diff_scale * kf * P.inv_h[1] * P.inv_h[1];
      fyf[f] = (float)fy[f];
    } else {
      long long f = e - nfx - nfy;
      int i = (int)(f % P.nx);
      long long t = f / P.nx;
      int j = (int)(t % P.ny), l = (int)(t / P.ny);
      double kf = l == 0 ? kap(i, j, 0) : l == P.nz ? kap(i, j, P.nz - 1) : hm(kap(i, j, l - 1), kap(i, j, l));
      // no diffusion along the time axis of a space-time problem
      fz[f] = P.time_axis ? 0.0 : diff_scale * kf * P.inv_h[2] * P.inv_h[2];
      fzf[f] = (float)fz[f];
    }
  }
}

template <int DIM>
__global__ void k_diag_shared(OpParams P, double *dinv, float *dinv32) {
  double cb[3] = {0, 0, 0};
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < P.N;
       g += (long long)gridDim.x * blockDim.x) {
    int i = (int)(g % P.nx);
    long long t = g / P.nx;
    int j = (int)(t % P.ny), l = (int)(t / P.ny);
    double d = 1.0 / diag_S<DIM>(P, cb, i, j, l);
    dinv[g] = d;
    dinv32[g] = (float)d;
  }
}

// ---------------------------------------------------------------------------
// Outer-iteration set-up (App. B.1 lines 3-5): r = b = rhs_I - S_IA psi_A,
// x = 0, per-instance Jacobi diagonal (convection), ||b||^2, |A|.  With a
// given start (x0 != null) the first outer iteration starts from x0 and each
// later one from the previous iterate y_prev, both restricted to I;
// k_start_resid then replaces r by b - S_II x.

template <int DIM, class V>
__global__ void __launch_bounds__(NT) k_outer_setup(OpParams P, const double *inst,
                                                    const double *psi, const uint8_t *mask,
                                                    V *r, double *b64, double *x, V *dinv,
                                                    InstState *st, double *part, int *cnt,
                                                    Ctrl *ctrl, int GX, const double *x0,
                                                    const double *y_prev) {
  __shared__ TileSmem<DIM, double> sm;
  __shared__ double red[NWARP];
  __shared__ double tot[2];
  __shared__ int flag;
  const int b = blockIdx.x, gblk = blockIdx.y;
  InstState &S = st[b];
  if (S.outer_done) return;
  const long long N = P.N;
  const double *ib = inst + 7 * b;
  double cb[3];
  inst_cb(P, ib, cb);
  const uint8_t *mk = mask + b * N;
  V *rb = r + b * N;
  double *bb64 = b64 + b * N, *xb = x + b * N;
  const double *x0b = x0 ? (S.outer == 0 ? x0 : y_prev) + b * N : nullptr;
  V *db = P.convection ? dinv + b * N : nullptr;
  double bb = 0.0, na = 0.0;
  const long long T = num_tiles<DIM>(P.nx, P.ny, P.nz);
  for (long long t = gblk; t < T; t += GX) {
    int ox, oy, oz;
    tile_origin<DIM>(P, t, ox, oy, oz);
    tile_S<DIM, double>(
        P, cb, ox, oy, oz, sm,
        [&](int, int, int, long long g) { return mk[g] ? psi[g] : 0.0; },
        [&](int, int gx, int gy, int gz, long long g, double su) {
          bool act = mk[g] != 0;
          double rhs = P.rhs ? P.rhs[b * N + g] : P.mass * desired(P, ib, gx, gy, gz);
          double bv = act ? 0.0 : rhs - su;
          bb64[g] = bv;
          rb[g] = (V)bv;
          xb[g] = (act || !x0b) ? 0.0 : x0b[g];
          if (db) db[g] = act ? (V)0 : (V)(1.0 / diag_S<DIM>(P, cb, gx, gy, gz));
          bb += bv * bv;
          na += act ? 1.0 : 0.0;
        });
  }
  bb = block_sum(bb, red);
  na = block_sum(na, red);
  if (threadIdx.x == 0) {
    part[(b * GX + gblk) * 2 + 0] = bb;
    part[(b * GX + gblk) * 2 + 1] = na;
  }
  if (!last_block(cnt + b * NCNT + CNT_SETUP, GX, &flag)) return;
  __shared__ double scratch[NT];
  reduce_fields(part + b * GX * 2, GX, 2, 2, tot, scratch);
  if (threadIdx.x == 0) {
    cnt[b * NCNT + CNT_SETUP] = 0;
    S.bnorm2 = tot[0];
    S.stats.n_active[S.outer] = (int)tot[1];
    S.empty_I = tot[1] >= (double)N ? 1 : 0;
    S.phase = 1;
    S.cg_done = 0;
    S.await = 0;
    S.stall = 0;
    S.floor2 = 0.0;
    S.rt2_prev = INFINITY;
    S.iters = 0;
    S.gamma = 0.0;
    S.beta = 0.0;
    S.csign = -1.0;
    S.rho = 0.0;
    S.sigma = 0.0;
    S.alpha = 1.0;
    for (int j = 0; j < SDF_MAX_K; ++j) S.t[j] = 0.0;
    atomicAdd(&ctrl->running, 1);
  }
}

// Residual of a given start: r = b - S_II x on I, 0 on A (x is zero on A),
// with the FP64 stencil.  Used only when the caller supplies x0.
template <int DIM, class V>
__global__ void __launch_bounds__(NT) k_start_resid(OpParams P, const double *inst,
                                                    const InstState *st, const uint8_t *mask,
                                                    const double *b64, const double *x, V *r,
                                                    int GX) {
  __shared__ TileSmem<DIM, double> sm;
  const int b = blockIdx.x, gblk = blockIdx.y;
  if (st[b].outer_done) return;
  const long long N = P.N;
  double cb[3];
  inst_cb(P, inst + 7 * b, cb);
  const uint8_t *mk = mask + b * N;
  const double *xb = x + b * N, *bb = b64 + b * N;
  V *rb = r + b * N;
  const long long T = num_tiles<DIM>(P.nx, P.ny, P.nz);
  for (long long t = gblk; t < T; t += GX) {
    int ox, oy, oz;
    tile_origin<DIM>(P, t, ox, oy, oz);
    tile_S<DIM, double>(
        P, cb, ox, oy, oz, sm, [&](int, int, int, long long g) { return xb[g]; },
        [&](int, int, int, int, long long g, double su) {
          rb[g] = mk[g] ? (V)0 : (V)(bb[g] - su);
        });
  }
}

// ---------------------------------------------------------------------------
// Coarse set-up (Sec. 2.2.1 Eq. coarse, Sec. 2.2.2): W_j = S_II (mask_I Phi_j)
// for one instance, then E_raw = Phi^T W and G = Phi^T diag(mask_I) Phi.

template <int DIM, class PhiT>
__global__ void __launch_bounds__(NT) k_modes_W(OpParams P, const double *inst, int b,
                                                const InstState *st, const uint8_t *mask,
                                                const PhiT *Phi, long long ld, double *W, int GX) {
  __shared__ TileSmem<DIM> sm;
  if (st[b].outer_done) return;
  const int j = blockIdx.x, gblk = blockIdx.y;
  const long long N = P.N;
  double cb[3];
  inst_cb(P, inst + 7 * b, cb);
  const uint8_t *mk = mask + b * N;
  const PhiT *ph = Phi + (long long)j * ld;
  double *wj = W + (long long)j * N;
  const long long T = num_tiles<DIM>(P.nx, P.ny, P.nz);
  for (long long t = gblk; t < T; t += GX) {
    int ox, oy, oz;
    tile_origin<DIM>(P, t, ox, oy, oz);
    tile_S<DIM>(
        P, cb, ox, oy, oz, sm, [&](int, int, int, long long g) { return mk[g] ? 0.0 : (double)ph[g]; },
        [&](int, int, int, int, long long g, double su) { wj[g] = mk[g] ? 0.0 : su; });
  }
}

// Tall-skinny Gram C = X^T diag(m) Y (k x k, FP64) with X = Phi and Y = W
// (which = 0) or Y = mask_I Phi (which = 1).  Per-block partials.
template <int KMAX, class PhiT>
__global__ void __launch_bounds__(NT) k_gram(const PhiT *Phi, long long ld, const double *W,
                                             const uint8_t *mask, const InstState *st, int b,
                                             long long N, int k, int which, double *gpart) {
  constexpr int MT = KMAX / 16, CH = 16;
  __shared__ double Xs[CH][KMAX + 1];
  __shared__ double Ys[CH][KMAX + 1];
  if (st[b].outer_done) return;
  const uint8_t *mk = mask + b * N;
  const int ti = threadIdx.x / 16, tj = threadIdx.x % 16;
  double acc[MT][MT];
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[a][c] = 0.0;
  for (long long base = (long long)blockIdx.x * CH; base < N; base += (long long)gridDim.x * CH) {
    for (int e = threadIdx.x; e < KMAX * CH; e += NT) {
      int c = e % CH, j = e / CH;
      long long g = base + c;
      double xv = 0.0, yv = 0.0;
      if (j < k && g < N) {
        xv = (double)Phi[(long long)j * ld + g];
        if (which == 0) yv = W[(long long)j * N + g];
        else yv = mk[g] ? 0.0 : xv;
      }
      Xs[c][j] = xv;
      Ys[c][j] = yv;
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < CH; ++c) {
      double xa[MT], yb[MT];
#pragma unroll
      for (int a = 0; a < MT; ++a) xa[a] = Xs[c][ti + 16 * a];
#pragma unroll
      for (int a = 0; a < MT; ++a) yb[a] = Ys[c][tj + 16 * a];
#pragma unroll
      for (int a = 0; a < MT; ++a)
#pragma unroll
        for (int q = 0; q < MT; ++q) acc[a][q] = fma(xa[a], yb[q], acc[a][q]);
    }
    __syncthreads();
  }
  double *out = gpart + (long long)blockIdx.x * k * k;
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int q = 0; q < MT; ++q) {
      int i = ti + 16 * a, j = tj + 16 * q;
      if (i < k && j < k) out[i * k + j] = acc[a][q];
    }
}

__global__ void k_gram_reduce(const double *gpart, int nblk, int k, const InstState *st, int b,
                              double *out) {
  if (st[b].outer_done) return;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  double s = 0.0;
  for (int g = 0; g < nblk; ++g) s += gpart[(long long)g * k * k + e];
  out[e] = s;
}

// Copy instance 0's E_raw and G to instances 1.. (one block per instance).
__global__ void k_coarse_copy(int k, double *Eraw, double *G) {
  const size_t kk = (size_t)k * k, b = blockIdx.x + 1;
  for (size_t e = threadIdx.x; e < kk; e += blockDim.x) {
    Eraw[b * kk + e] = Eraw[e];
    G[b * kk + e] = G[e];
  }
}

// k x k coarse factorisation for each instance (one block per instance):
//   G = L_g L_g^T (Cholesky-QR of Phi_I; rank test as in the oracle),
//   E = L_g^-1 E_raw L_g^-T  (the Galerkin matrix in the orthonormal basis),
//   E = L_e L_e^T, Einv_raw = F^T F with F = L_e^-1 L_g^-1,
//   cond(E) by power iteration on E and on E^-1 (guard, Remark tau_cond).
__device__ bool dev_cholesky(double *A, int k, double *red, int *ok_s, double rank_tol) {
  // left-looking, lower triangle of the row-major k x k matrix A (in place)
  double dmax = 0.0;
  for (int i = 0; i < k; ++i) dmax = fmax(dmax, A[i * k + i]);
  __syncthreads();  // every thread has read the diagonal before it changes
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      double d = A[j * k + j];
      for (int m = 0; m < j; ++m) d -= A[j * k + m] * A[j * k + m];
      *ok_s = (d > rank_tol * dmax) && isfinite(d);
      red[0] = (*ok_s) ? sqrt(d) : 1.0;
      A[j * k + j] = red[0];
    }
    __syncthreads();
    if (!*ok_s) return false;
    double d = red[0];
    for (int i = j + 1 + threadIdx.x; i < k; i += NT) {
      double s = A[i * k + j];
      for (int m = 0; m < j; ++m) s -= A[i * k + m] * A[j * k + m];
      A[i * k + j] = s / d;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < k * k; e += NT)
    if (e % k > e / k) A[e] = 0.0;  // clear the upper triangle
  __syncthreads();
  return true;
}

// Inverse of a lower-triangular row-major L into Li (thread per column).
__device__ void dev_tri_inv(const double *L, double *Li, int k) {
  for (int c = threadIdx.x; c < k; c += NT) {
    for (int i = 0; i < k; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      if (i >= c)
        for (int m = c; m < i; ++m) s -= L[i * k + m] * Li[m * k + c];
      Li[i * k + c] = (i >= c) ? s / L[i * k + i] : 0.0;
    }
  }
  __syncthreads();
}

// C = A B (row-major k x k), transA / transB select A^T / B^T.
__device__ void dev_gemm(const double *A, const double *B, double *C, int k, bool tA, bool tB) {
  for (int e = threadIdx.x; e < k * k; e += NT) {
    int i = e / k, j = e % k;
    double s = 0.0;
    for (int m = 0; m < k; ++m) {
      double a = tA ? A[m * k + i] : A[i * k + m];
      double bb = tB ? B[j * k + m] : B[m * k + j];
      s = fma(a, bb, s);
    }
    C[e] = s;
  }
  __syncthreads();
}

// largest eigenvalue of the SPD operator v -> M v (M given by up to two
// triangular factors: op 0: M = E; op 1: M = Li^T Li), power iteration.
__device__ double dev_power(const double *E, const double *Li, int k, int op, double *v,
                            double *w, double *red) {
  for (int i = threadIdx.x; i < k; i += NT) v[i] = 1.0 + 0.5 * sin((double)(i + 1));
  __syncthreads();
  double lam = 0.0;
  for (int it = 0; it < 120; ++it) {
    // w = M v
    for (int i = threadIdx.x; i < k; i += NT) {
      double s = 0.0;
      if (op == 0) {
        for (int m = 0; m < k; ++m) s = fma(E[i * k + m], v[m], s);
      } else {
        for (int m = 0; m <= i; ++m) s = fma(Li[i * k + m], v[m], s);  // Li v
      }
      w[i] = s;
    }
    __syncthreads();
    if (op == 1) {  // v2 = Li^T w, stored in v
      for (int i = threadIdx.x; i < k; i += NT) {
        double s = 0.0;
        for (int m = i; m < k; ++m) s = fma(Li[m * k + i], w[m], s);
        v[i] = s;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < k; i += NT) w[i] = v[i];
      __syncthreads();
    }
    double nn = 0.0;
    for (int i = threadIdx.x; i < k; i += NT) nn += w[i] * w[i];
    nn = block_sum(nn, red);
    double nrm = sqrt(nn);
    lam = nrm;  // ||M v|| with ||v|| = 1 after the first step
    for (int i = threadIdx.x; i < k; i += NT) v[i] = nrm > 0 ? w[i] / nrm : 0.0;
    __syncthreads();
  }
  return lam;
}

// host_decides = 1: the deflation decision is left to a host step that works
// from G and E_raw alone (the safe merge); the factorisations may then fail.
__global__ void __launch_bounds__(NT) k_coarse(int k, InstState *st, const double *G,
                                               const double *Eraw, double *Einv, double *wk,
                                               double tau_cond, int host_decides) {
  __shared__ double red[NWARP];
  __shared__ int ok;
  __shared__ double vv[SDF_MAX_K], ww[SDF_MAX_K];
  const int b = blockIdx.x;
  InstState &S = st[b];
  if (S.outer_done) return;
  const size_t kk = (size_t)k * k;
  double *Lg = wk + (size_t)b * 5 * kk, *Lgi = Lg + kk, *T = Lgi + kk, *E = T + kk, *Lei = E + kk;
  const double *Gb = G + (size_t)b * kk, *Eb = Eraw + (size_t)b * kk;
  double *Ei = Einv + (size_t)b * kk;
  if (S.empty_I) {  // n_I = 0: nothing to solve, no guard decision (as the oracle)
    if (threadIdx.x == 0) {
      S.deflate = 0;
      S.stats.cond_E[S.outer] = 0.0;
      S.stats.fallback[S.outer] = 0;
    }
    return;
  }
  for (size_t e = threadIdx.x; e < kk; e += NT) Lg[e] = Gb[e];
  __syncthreads();
  bool good = dev_cholesky(Lg, k, red, &ok, 1e-14);  // rank test: R_jj^2 <= 1e-14 max R^2
  double cond = INFINITY;
  if (good) {
    dev_tri_inv(Lg, Lgi, k);
    dev_gemm(Lgi, Eb, T, k, false, false);  // T = Lg^-1 Eraw
    dev_gemm(T, Lgi, E, k, false, true);    // E = T Lg^-T
    for (size_t e = threadIdx.x; e < kk; e += NT) {
      int i = (int)(e / k), j = (int)(e % k);
      if (i < j) {
        double s = 0.5 * (E[i * k + j] + E[j * k + i]);
        E[i * k + j] = s;
        E[j * k + i] = s;
      }
    }
    __syncthreads();
    double lmax = dev_power(E, nullptr, k, 0, vv, ww, red);
    for (size_t e = threadIdx.x; e < kk; e += NT) T[e] = E[e];
    __syncthreads();
    good = dev_cholesky(T, k, red, &ok, 0.0);
    if (good) {
      dev_tri_inv(T, Lei, k);
      double linv = dev_power(nullptr, Lei, k, 1, vv, ww, red);  // lambda_max(E^-1)
      cond = (linv > 0 && lmax > 0) ? lmax * linv : INFINITY;
      if (cond <= tau_cond) {
        dev_gemm(Lei, Lgi, T, k, false, false);  // F = Le^-1 Lg^-1
        dev_gemm(T, T, Ei, k, true, false);      // Einv_raw = F^T F
      } else {
        good = false;
      }
    }
  }
  if (threadIdx.x == 0) {
    S.deflate = (good || host_decides) ? 1 : 0;
    S.stats.cond_E[S.outer] = cond;
    S.stats.fallback[S.outer] = good ? 0 : 1;
  }
}

// ---------------------------------------------------------------------------
// Projection t = Phi_I^T v (initial coarse correction and sdf_project).

template <int KMAX, class PhiT, class V>
__global__ void __launch_bounds__(NT) k_project(const PhiT *Phi, long long ld, int k, long long N,
                                                const uint8_t *mask, const V *v,
                                                InstState *st, double *out, double *part,
                                                int *cnt, int GX) {
  __shared__ V vs[512];
  __shared__ double scratch[NT];
  __shared__ int flag;
  const int b = blockIdx.x, gblk = blockIdx.y;
  if (st) {
    const InstState &S = st[b];
    if (S.outer_done || S.cg_done || !S.deflate) return;
  }
  const uint8_t *mk = mask + b * N;
  const V *vb = v + b * N;
  double acc[KMAX / NWARP];
#pragma unroll
  for (int a = 0; a < KMAX / NWARP; ++a) acc[a] = 0.0;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (long long base = (long long)gblk * 512; base < N; base += (long long)GX * 512) {
    for (int e = threadIdx.x; e < 512; e += NT) {
      long long g = base + e;
      vs[e] = (g < N && !mk[g]) ? vb[g] : (V)0;
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < KMAX / NWARP; ++a) {
      int j = warp + NWARP * a;
      if (j < k) {
        const PhiT *ph = Phi + (long long)j * ld + base;
        V s = (V)0;
        for (int e = lane; e < 512; e += 32)
          if (base + e < N) s = fma((V)ph[e], vs[e], s);
        acc[a] += (double)s;
      }
    }
    __syncthreads();
  }
  const int F = KMAX;
  double *pb = part + ((long long)b * GX + gblk) * F;
#pragma unroll
  for (int a = 0; a < KMAX / NWARP; ++a) {
    double s = warp_sum(acc[a]);
    int j = warp + NWARP * a;
    if (lane == 0 && j < k) pb[j] = s;
  }
  if (!last_block(cnt + b * NCNT + CNT_PROJECT, GX, &flag)) return;
  __shared__ double res[SDF_MAX_K];
  reduce_fields(part + (long long)b * GX * F, GX, F, k, res, scratch);
  if (threadIdx.x == 0) cnt[b * NCNT + CNT_PROJECT] = 0;
  for (int j = threadIdx.x; j < k; j += NT) {
    if (st) st[b].t[j] = res[j];
    else out[b * k + j] = res[j];
  }
}

// ---------------------------------------------------------------------------
// CG iteration, kernel A: p = mask_I (gamma D^-1 r - Phi c + beta p) with
// c = csign E_raw^-1 t (the coarse GEMV, recomputed by every block).

template <int KMAX, class PhiT, class V>
__global__ void __launch_bounds__(NT) k_expand(const PhiT *Phi, long long ld, int k, long long N,
                                               const InstState *st, const double *Einv,
                                               const uint8_t *mask, const V *r, const V *dinv,
                                               int dinv_per_inst, V *p, int GX) {
  __shared__ V c[SDF_MAX_K];
  const int b = blockIdx.x, gblk = blockIdx.y;
  const InstState &S = st[b];
  if (S.outer_done || S.cg_done || (S.await && S.phase == 0)) return;
  const int defl = S.deflate;
  const V gam = (V)S.gamma, bet = (V)S.beta;
  if (defl) {
    const double *Ei = Einv + (size_t)b * k * k;
    for (int i = threadIdx.x; i < k; i += NT) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s = fma(Ei[i * k + j], S.t[j], s);
      c[i] = (V)(S.csign * s);
    }
  }
  __syncthreads();
  const uint8_t *mk = mask + b * N;
  const V *rb = r + b * N;
  const V *db = dinv + (dinv_per_inst ? b * N : 0);
  V *pb = p + b * N;
  for (long long g = (long long)gblk * NT + threadIdx.x; g < N; g += (long long)GX * NT) {
    V v = (V)0;
    if (!mk[g]) {
      v = gam * db[g] * rb[g];
      if (bet != (V)0) v += bet * pb[g];  // p is not read on the first pass (never written)
      if (defl) {
        V s0 = (V)0, s1 = (V)0;
        int j = 0;
        for (; j + 1 < k; j += 2) {
          s0 = fma((V)Phi[(long long)j * ld + g], c[j], s0);
          s1 = fma((V)Phi[(long long)(j + 1) * ld + g], c[j + 1], s1);
        }
        if (j < k) s0 = fma((V)Phi[(long long)j * ld + g], c[j], s0);
        v -= s0 + s1;
      }
    }
    pb[g] = v;
  }
}

// Kernel B: q = S_II p and sigma = (p, q) (FP64 accumulation); the last
// block sets alpha (1 in the coarse and correction passes).
template <int DIM, class V>
__global__ void __launch_bounds__(NT) k_spmv(OpParams P, const double *inst, InstState *st,
                                             const uint8_t *mask, const V *p, V *q,
                                             double *part, int *cnt, Ctrl *ctrl, int GX) {
  __shared__ TileSmem<DIM, V> sm;
  __shared__ double red[NWARP];
  __shared__ int flag;
  const int b = blockIdx.x, gblk = blockIdx.y;
  InstState &S = st[b];
  if (S.outer_done || S.cg_done || (S.await && S.phase == 0)) return;
  const long long N = P.N;
  double cb[3];
  inst_cb(P, inst + 7 * b, cb);
  const uint8_t *mk = mask + b * N;
  const V *pb = p + b * N;
  V *qb = q + b * N;
  double sg = 0.0;
  KahanF sgf;  // FP32 path: compensated FP32 sum, FP64 across threads
  const long long T = num_tiles<DIM>(P.nx, P.ny, P.nz);
  for (long long t = gblk; t < T; t += GX) {
    int ox, oy, oz;
    tile_origin<DIM>(P, t, ox, oy, oz);
    tile_S<DIM, V>(
        P, cb, ox, oy, oz, sm, [&](int, int, int, long long g) { return pb[g]; },
        [&](int e, int, int, int, long long g, V su) {
          V qv = mk[g] ? (V)0 : su;
          qb[g] = qv;
          V pv;
          if constexpr (DIM == 1) {  // CSR rows: no staged halo, p from memory
            pv = pb[g];
          } else {
            pv = sm.u[uidx<DIM>(e % TileCfg<DIM>::TX, (e / TileCfg<DIM>::TX) % TileCfg<DIM>::TY,
                                e / (TileCfg<DIM>::TX * TileCfg<DIM>::TY))];
          }
          if constexpr (sizeof(V) == sizeof(float)) sgf.add(pv * qv);
          else sg = fma((double)pv, (double)qv, sg);
        });
  }
  if constexpr (sizeof(V) == sizeof(float)) sg = sgf.value();
  sg = block_sum(sg, red);
  if (threadIdx.x == 0) part[b * GX + gblk] = sg;
  if (!last_block(cnt + b * NCNT + CNT_SIGMA, GX, &flag)) return;
  __shared__ double scratch[NT];
  __shared__ double tot1[1];
  reduce_fields(part + (long long)b * GX, GX, 1, 1, tot1, scratch);
  if (threadIdx.x == 0) {
    double s = tot1[0];
    cnt[b * NCNT + CNT_SIGMA] = 0;
    S.sigma = s;
    if (S.phase) {
      S.alpha = 1.0;
    } else if (s > 0.0 && isfinite(s)) {
      S.alpha = S.rho / s;
    } else {
      S.stats.status = isfinite(s) ? SDF_ERR_BREAKDOWN : SDF_ERR_NONFINITE;
      S.cg_done = 1;
      S.stats.cg_iters[S.outer] = S.iters;
      atomicSub(&ctrl->running, 1);
    }
  }
}

// Kernel C: x += alpha p (x in FP64), r -= alpha q, z = D^-1 r, v = S_II z - r,
// t = Phi_I^T v, rho = (r, z), ||r||^2 (FP64 accumulation); the last block
// tests convergence (App. B.2) and prepares beta for kernel A.  r is read
// (with its halo) from r_in and written to r_out: blocks read neighbouring
// tiles' r while other blocks update theirs, so the update cannot be in place.
// Passes: phase 0 = CG iteration; 1 = coarse-corrected start (beta = 0);
// 2 = coarse correction after an FP64 residual replacement (beta continues).
// mixed = 1: convergence is only declared by the FP64 check of k_resid; the
// recurrence reaching rtol sets `await` instead.
template <int DIM, int KMAX, class PhiT, class V>
__global__ void __launch_bounds__(NT) k_update(OpParams P, const double *inst, const PhiT *Phi,
                                               long long ld, int k, InstState *st,
                                               const uint8_t *mask, const V *r_in, V *r_out,
                                               const V *q, const V *p, double *x, const V *dinv,
                                               double *part, int *cnt, Ctrl *ctrl, int GX,
                                               double rtol2, int max_cg, int mixed, V *vout) {
  __shared__ TileSmem<DIM, V> sm;
  __shared__ double red[NWARP];
  __shared__ double scratch[NT];
  __shared__ double res[SDF_MAX_K + 2];
  __shared__ int flag;
  const int b = blockIdx.x, gblk = blockIdx.y;
  InstState &S = st[b];
  if (S.outer_done || S.cg_done || (S.await && S.phase == 0)) return;
  const long long N = P.N;
  const double alpha64 = S.alpha;
  const V alpha = (V)alpha64;
  // vout: v = S z - r is written for the batch projection GEMM instead of
  // being projected here (shared-Phi batch kernels)
  const int defl = vout ? 0 : S.deflate;
  V *vb = vout ? vout + b * N : nullptr;
  double cb[3];
  inst_cb(P, inst + 7 * b, cb);
  const uint8_t *mk = mask + b * N;
  const V *rb = r_in + b * N;
  V *rw = r_out + b * N;
  double *xb = x + b * N;
  const V *qb = q + b * N, *pb = p + b * N;
  const V *db = dinv + (P.convection ? b * N : 0);
  double rho = 0.0, rr = 0.0;
  // FP64 path: warp-per-mode projection of the tile (tile_project).
  // FP32 path: every thread accumulates Phi_j(g) v(g) for its own nodes and
  // all modes in registers (coalesced, many independent loads in flight).
  constexpr bool kThreadProj = sizeof(V) == sizeof(float);
  constexpr int NACC = kThreadProj ? KMAX : KMAX / NWARP;
  double acc[kThreadProj ? 1 : KMAX / NWARP];
  float accf[kThreadProj ? KMAX : 1];
#pragma unroll
  for (int a = 0; a < (kThreadProj ? 1 : KMAX / NWARP); ++a) acc[a] = 0.0;
#pragma unroll
  for (int a = 0; a < (kThreadProj ? KMAX : 1); ++a) accf[a] = 0.0f;
  const long long T = num_tiles<DIM>(P.nx, P.ny, P.nz);
  for (long long t = gblk; t < T; t += GX) {
    int ox, oy, oz;
    tile_origin<DIM>(P, t, ox, oy, oz);
    tile_S<DIM, V>(
        P, cb, ox, oy, oz, sm,
        [&](int, int, int, long long g) {
          return mk[g] ? (V)0 : db[g] * (rb[g] - alpha * qb[g]);
        },
        [&](int e, int, int, int, long long g, V su) {
          if (mk[g]) {
            sm.v[e] = (V)0;
            rw[g] = (V)0;
            if (vb) vb[g] = (V)0;
            return;
          }
          V rn = rb[g] - alpha * qb[g];
          V z = db[g] * rn;
          xb[g] = fma(alpha64, (double)pb[g], xb[g]);
          rw[g] = rn;
          rho = fma((double)rn, (double)z, rho);
          rr = fma((double)rn, (double)rn, rr);
          // A-DEF2 (P^T M^-1 + Q): the next direction is z - Phi E^-1 Phi_I^T (S z - r);
          // the Q r part vanishes in exact arithmetic but keeps the coarse-space
          // component that rounding feeds into r out of the iteration
          sm.v[e] = su - rn;
          if (vb) vb[g] = su - rn;
          if constexpr (kThreadProj) {
            if (defl) {
#pragma unroll
              for (int j = 0; j < KMAX; ++j)
                if (j < k)
                  accf[j] = fmaf((float)Phi[(long long)j * ld + g], (float)(su - rn), accf[j]);
            }
          }
        });
    if constexpr (!kThreadProj) {
      if (defl) {
        tile_project<DIM, KMAX>(P, Phi, ld, k, ox, oy, oz, sm.v, acc);
        __syncthreads();
      }
    }
  }
  (void)NACC;
  rho = block_sum(rho, red);
  rr = block_sum(rr, red);
  const int F = KMAX + 2;
  double *pbk = part + ((long long)b * GX + gblk) * F;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (defl) {
    if constexpr (kThreadProj) {
      block_sum_modes<KMAX>(accf, k, pbk + 2, scratch);
    } else {
#pragma unroll
      for (int a = 0; a < KMAX / NWARP; ++a) {
        double sacc = warp_sum(acc[a]);
        int j = warp + NWARP * a;
        if (lane == 0 && j < k) pbk[2 + j] = sacc;
      }
    }
  }
  if (threadIdx.x == 0) {
    pbk[0] = rho;
    pbk[1] = rr;
  }
  if (!last_block(cnt + b * NCNT + CNT_UPDATE, GX, &flag)) return;
  reduce_fields(part + (long long)b * GX * F, GX, F, defl ? 2 + k : 2, res, scratch);
  if (defl)
    for (int j = threadIdx.x; j < k; j += NT) S.t[j] = res[2 + j];
  if (threadIdx.x == 0) {
    cnt[b * NCNT + CNT_UPDATE] = 0;
    double rho_new = res[0], rn2 = res[1];
    if (S.phase == 0) S.iters += 1;
    S.rnorm2 = rn2;
    bool conv = rn2 <= rtol2 * S.bnorm2;
    if (!isfinite(rho_new) || !isfinite(rn2)) {
      S.stats.status = SDF_ERR_NONFINITE;
      S.cg_done = 1;
    } else if (conv && !mixed) {
      S.cg_done = 1;
    } else if (S.iters >= max_cg) {
      S.stats.status = SDF_ERR_CG_MAXIT;
      S.cg_done = 1;
    } else {
      if (conv) S.await = 1;
      // A correction pass (phase 2) replaces the residual of the iteration
      // that preceded it, so its beta divides by that iteration's old rho.
      S.beta = S.phase == 1 ? 0.0 : rho_new / (S.phase == 2 ? S.rho_prev : S.rho);
      if (S.phase != 2) S.rho_prev = S.rho;
      S.rho = rho_new;
      S.gamma = 1.0;
      S.csign = 1.0;
      S.phase = 0;
    }
    if (S.cg_done) {
      S.stats.cg_iters[S.outer] = S.iters;
      S.stats.relres[S.outer] = S.bnorm2 > 0 ? sqrt(rn2 / S.bnorm2) : 0.0;
      atomicSub(&ctrl->running, 1);
    }
  }
}

// Checkerboard sign s_g = (-1)^(i+j+l) of a grid node.  A couples nearest
// neighbours only (upwind and time terms included), so its graph is
// bipartite, and it is an M-matrix (positive diagonal, non-positive
// off-diagonals).  Every entry of S = mass I + w A^T A then has the sign
// s_i s_j: |S| = D_s S D_s with D_s = diag(s), so the product with the
// entrywise absolute value is |S_II| |x| = s o (S_II (s o |x|)) and its norm is
// that of the ordinary (sign-free, cancellation-free) product S_II (s o |x|).
__device__ __forceinline__ double signed_abs(int gx, int gy, int gz, double v) {
  return ((gx + gy + gz) & 1) ? -fabs(v) : fabs(v);
}

// FP64 residual replacement of the mixed path: r = b - S_II x with the FP64
// stencil on the FP64 iterate and ||r||^2.  The last block declares
// convergence on this true residual when ||r|| <= max(rtol ||b||, floor) with
// floor = floor_c u || |S_II||x| || (the attainable accuracy of an FP64
// residual, App. B.2's recurrence stop read for a method whose recurrence runs
// in FP32), or arms the coarse correction pass (phase 2: w = Phi E_raw^-1
// Phi_I^T r, alpha = 1) whose projection the GEMM computes from the new r.
// The floor is evaluated (a second stencil pass on s o |x|) once per solve:
// at the first replacement where the recurrence has met rtol or the true
// residual stalled (it fell less than 2x while the recurrence ran more than
// 10x below it); near convergence x, and with it the floor, barely moves.  r is written in place: this
// kernel reads x, not r.
// FP64 column-stencil source and output of the 3D residual replacement:
// u = x + x_lo, r = b - S_II u (FP32 copy, zero on the active set), ||r||^2.
struct ColSrcX {
  static constexpr bool AUX = false;
  const double *x;
  const float *xl;
  struct Raw { double x; float l; };
  __device__ __forceinline__ Raw fetch(int g) const { return Raw{x[g], xl[g]}; }
  __device__ __forceinline__ double value(const Raw &a) const { return a.x + (double)a.l; }
};
struct ColOutResid {
  const uint8_t *mk;
  const double *b;
  float *r;
  double rr;
  struct Pre { double b; uint8_t m; };
  __device__ __forceinline__ Pre fetch(int g) const { return Pre{b[g], mk[g]}; }
  __device__ __forceinline__ void store(int g, double su, double, double, const Pre &a) {
    if (a.m) {
      r[g] = 0.0f;
      return;
    }
    const double rt = a.b - su;
    r[g] = (float)rt;
    rr = fma(rt, rt, rr);
  }
};

template <int DIM>
__global__ void __launch_bounds__(NT) k_resid(OpParams P, const double *inst, InstState *st,
                                              const uint8_t *mask, const double *b64,
                                              const double *x, const float *xlo, float *r,
                                              double *part, int *cnt, Ctrl *ctrl, int GX,
                                              double rtol2, double floor_cu, int zc) {
  // 3D: the residual by the z-marching column stencil (u loaded 1.4 and w
  // computed 1.2 times per node, against 4.5 and 2.4 on halo-2 tiles); the
  // floor pass, once per solve, on tiles.  The two share one buffer.
  constexpr size_t kSm = (DIM == 3 && sizeof(ColSmem<double>) > sizeof(TileSmem<DIM, double>))
                             ? sizeof(ColSmem<double>)
                             : sizeof(TileSmem<DIM, double>);
  __shared__ __align__(16) unsigned char smraw[kSm];
  TileSmem<DIM, double> &sm = *reinterpret_cast<TileSmem<DIM, double> *>(smraw);
  __shared__ double red[NWARP];
  __shared__ int flag;
  const int b = blockIdx.x, gblk = blockIdx.y;
  InstState &S = st[b];
  if (S.outer_done || S.cg_done) return;
  // the floor is evaluated once per solve, when first needed (uniform in the block)
  const bool need_floor = floor_cu > 0.0 && S.floor2 == 0.0 && (S.await || S.stall);
  const long long N = P.N;
  double cb[3];
  inst_cb(P, inst + 7 * b, cb);
  const uint8_t *mk = mask + b * N;
  const double *xb = x + b * N, *bb = b64 + b * N;
  const float *xl = xlo + b * N;
  float *rb = r + b * N;
  double rr = 0.0, ff = 0.0;
  const long long T = num_tiles<DIM>(P.nx, P.ny, P.nz);
  if constexpr (DIM == 3) {  // the mixed path has no convection
    ColSmem<double> &cs = *reinterpret_cast<ColSmem<double> *>(smraw);
    const ColSrcX src{xb, xl};
    ColOutResid out{mk, bb, rb, 0.0};
    const long long items = col_items(P.nx, P.ny, P.nz, zc);
    for (long long t = gblk; t < items; t += GX) {
      int x0, y0, z0, z1;
      col_origin(P, t, zc, x0, y0, z0, z1);
      if (P.fx)
        col_S3<double, true, false>(P, cb, x0, y0, z0, z1, cs, src, out);
      else
        col_S3<double, false, false>(P, cb, x0, y0, z0, z1, cs, src, out);
    }
    rr = out.rr;
  } else {
    for (long long t = gblk; t < T; t += GX) {
      int ox, oy, oz;
      tile_origin<DIM>(P, t, ox, oy, oz);
      tile_S<DIM, double>(
          P, cb, ox, oy, oz, sm,
          [&](int, int, int, long long g) { return xb[g] + (double)xl[g]; },
          [&](int, int, int, int, long long g, double su) {
            if (mk[g]) {
              rb[g] = 0.0f;
              return;
            }
            const double rt = bb[g] - su;
            rb[g] = (float)rt;
            rr = fma(rt, rt, rr);
          });
    }
  }
  for (long long t = gblk; need_floor && t < T; t += GX) {
    int ox, oy, oz;
    tile_origin<DIM>(P, t, ox, oy, oz);
    tile_S<DIM, double>(
        P, cb, ox, oy, oz, sm,
        [&](int gx, int gy, int gz, long long g) {
          return mk[g] ? 0.0 : signed_abs(gx, gy, gz, xb[g] + (double)xl[g]);
        },
        [&](int, int, int, int, long long g, double su) {
          if (!mk[g]) ff = fma(su, su, ff);
        });
  }
  rr = block_sum(rr, red);
  ff = block_sum(ff, red);
  if (threadIdx.x == 0) {
    part[((long long)b * GX + gblk) * 2 + 0] = rr;
    part[((long long)b * GX + gblk) * 2 + 1] = ff;
  }
  if (!last_block(cnt + b * NCNT + CNT_UPDATE, GX, &flag)) return;
  __shared__ double scratch[NT];
  __shared__ double tot2[2];
  reduce_fields(part + (long long)b * GX * 2, GX, 2, 2, tot2, scratch);
  if (threadIdx.x == 0) {
    const double rn2 = tot2[0];
    const double rec2 = S.rnorm2;  // the recurrence residual this replaces
    cnt[b * NCNT + CNT_UPDATE] = 0;
    S.rnorm2 = rn2;
    if (need_floor) S.floor2 = floor_cu * floor_cu * tot2[1];
    const double rtb = rtol2 * S.bnorm2;
    if (!isfinite(rn2)) {
      S.stats.status = SDF_ERR_NONFINITE;
      S.cg_done = 1;
    } else if (rn2 <= fmax(rtb, S.floor2)) {
      S.cg_done = 1;
      S.stats.floor_stop[S.outer] = rn2 > rtb ? 1 : 0;
    } else {
      // stalled: the true residual fell less than 2x since the last
      // replacement while the recurrence ran more than 10x below it (the
      // drift of a residual at its attainable accuracy)
      S.stall = (rn2 > 0.25 * S.rt2_prev && rec2 < 0.01 * rn2) ? 1 : 0;
      S.await = 0;
      S.phase = 2;
      S.gamma = 0.0;
      S.beta = 0.0;
      S.csign = -1.0;
    }
    S.rt2_prev = rn2;
    if (S.cg_done) {
      S.stats.cg_iters[S.outer] = S.iters;
      S.stats.relres[S.outer] = S.bnorm2 > 0 ? sqrt(rn2 / S.bnorm2) : 0.0;
      atomicSub(&ctrl->running, 1);
    }
  }
}

// True residual and attainable-accuracy floor of each instance's final inner
// solve (App. B.2; see sdf_stats), both paths: ||b - S_II x||^2 and
// || |S_II||x| ||^2 in FP64 (x = x + x_lo on the mixed path), the latter as
// S_II (s o |x|) on a grid (signed_abs) and with |S| row by row on a problem
// given by its operator.
template <int DIM>
__global__ void __launch_bounds__(NT) k_exit_resid(OpParams P, const double *inst, InstState *st,
                                                   const uint8_t *mask, const double *b64,
                                                   const double *x, const float *xlo,
                                                   double *part, int *cnt, int GX,
                                                   double floor_cu) {
  __shared__ TileSmem<DIM, double> sm;
  __shared__ double red[NWARP];
  __shared__ int flag;
  const int b = blockIdx.x, gblk = blockIdx.y;
  InstState &S = st[b];
  if (S.outer_done) return;
  const long long N = P.N;
  double cb[3];
  inst_cb(P, inst + 7 * b, cb);
  const uint8_t *mk = mask + b * N;
  const double *xb = x + b * N, *bb = b64 + b * N;
  const float *xl = xlo ? xlo + b * N : nullptr;
  auto xval = [&](long long g) { return mk[g] ? 0.0 : (xl ? xb[g] + (double)xl[g] : xb[g]); };
  double rr = 0.0, ff = 0.0;
  const long long T = num_tiles<DIM>(P.nx, P.ny, P.nz);
  for (long long t = gblk; t < T; t += GX) {
    int ox, oy, oz;
    tile_origin<DIM>(P, t, ox, oy, oz);
    tile_S<DIM, double>(
        P, cb, ox, oy, oz, sm, [&](int, int, int, long long g) { return xval(g); },
        [&](int, int, int, int, long long g, double su) {
          if (mk[g]) return;
          const double rt = bb[g] - su;
          rr = fma(rt, rt, rr);
        });
    if constexpr (DIM == 1) {  // |S| x row by row from the assembled CSR S
      for (int e = threadIdx.x; e < TileCfg<1>::TX; e += NT) {
        const long long g = ox + e;
        if (g >= N || mk[g]) continue;
        double acc = 0.0;
        for (int q = P.csr_rp[g], qe = P.csr_rp[g + 1]; q < qe; ++q)
          acc = fma(fabs(P.csr_v[q]), fabs(xval(P.csr_ci[q])), acc);
        ff = fma(acc, acc, ff);
      }
    } else {
      tile_S<DIM, double>(
          P, cb, ox, oy, oz, sm,
          [&](int gx, int gy, int gz, long long g) { return signed_abs(gx, gy, gz, xval(g)); },
          [&](int, int, int, int, long long g, double su) {
            if (!mk[g]) ff = fma(su, su, ff);
          });
    }
  }
  rr = block_sum(rr, red);
  ff = block_sum(ff, red);
  if (threadIdx.x == 0) {
    part[((long long)b * GX + gblk) * 2 + 0] = rr;
    part[((long long)b * GX + gblk) * 2 + 1] = ff;
  }
  if (!last_block(cnt + b * NCNT + CNT_SETUP, GX, &flag)) return;
  __shared__ double scratch[NT];
  __shared__ double tot2[2];
  reduce_fields(part + (long long)b * GX * 2, GX, 2, 2, tot2, scratch);
  if (threadIdx.x == 0) {
    cnt[b * NCNT + CNT_SETUP] = 0;
    const bool has_b = S.bnorm2 > 0.0;
    S.stats.true_relres[S.outer] = has_b ? sqrt(tot2[0] / S.bnorm2) : 0.0;
    S.stats.relres_floor[S.outer] = has_b ? floor_cu * sqrt(tot2[1] / S.bnorm2) : 0.0;
  }
}

// ---------------------------------------------------------------------------
// Mixed path, shared-Phi kernels.  The per-instance stencil work (k_spmv,
// k_update_v) runs on tiles; everything that reads Phi reads it once per
// launch for all instances of the batch: the expansion keeps one node's k mode
// values in registers and applies them to every instance, and the projection
// is a tall-skinny GEMM T = Phi^T [v_1 ... v_B] over shared-memory chunks.

// Instance b takes part in the current pass.
__device__ __forceinline__ bool inst_running(const InstState &S) {
  return !(S.outer_done || S.cg_done || (S.await && S.phase == 0));
}

// p_b = mask_I (gamma_b D^-1 r_b - Phi c_b + beta_b p_b) for every running
// instance.  Dynamic shared memory: c (B x KMAX floats), gamma, beta, flags.
template <int KMAX, class PhiT>
__global__ void __launch_bounds__(NT) k_expand_b(const PhiT *__restrict__ Phi, long long ld, int k,
                                                 long long N, int B, const InstState *st,
                                                 const float *cvec, const uint8_t *mask,
                                                 const float *r, const float *dinv,
                                                 int dinv_per_inst, float *p) {
  extern __shared__ float dsm[];
  float *cs = dsm;
  float *gam = cs + (size_t)B * KMAX;
  float *bet = gam + B;
  int *act = (int *)(bet + B);
  for (int b = threadIdx.x; b < B; b += NT) {
    const InstState &S = st[b];
    act[b] = inst_running(S) ? (1 | (S.deflate ? 2 : 0)) : 0;
    gam[b] = (float)S.gamma;
    bet[b] = (float)S.beta;
  }
  for (int e = threadIdx.x; e < B * KMAX; e += NT) cs[e] = cvec[e];
  __syncthreads();
  for (long long g = (long long)blockIdx.x * NT + threadIdx.x; g < N;
       g += (long long)gridDim.x * NT) {
    float ph[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) ph[j] = j < k ? (float)Phi[(long long)j * ld + g] : 0.0f;
    const float d_shared = dinv_per_inst ? 0.0f : dinv[g];
    // instances in groups of four: every load of the group is issued before
    // the mode sums, so the memory latency of one instance overlaps the others
    for (int b0 = 0; b0 < B; b0 += 4) {
      uint8_t mk[4];
      float dv[4], rv[4], pv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int b = b0 + u;
        const bool on = b < B && act[b];
        const long long gb = (long long)b * N + g;
        mk[u] = on ? mask[gb] : (uint8_t)1;
        dv[u] = on ? (dinv_per_inst ? dinv[gb] : d_shared) : 0.0f;
        rv[u] = on ? r[gb] : 0.0f;
        pv[u] = (on && bet[b] != 0.0f) ? p[gb] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int b = b0 + u;
        if (b >= B || !act[b]) continue;
        float v = 0.0f;
        if (!mk[u]) {
          v = fmaf(bet[b], pv[u], gam[b] * dv[u] * rv[u]);
          if (act[b] & 2) {
            const float *cb = cs + (size_t)b * KMAX;
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int j = 0; j < KMAX; j += 2) {
              s0 = fmaf(ph[j], cb[j], s0);
              s1 = fmaf(ph[j + 1], cb[j + 1], s1);
            }
            v -= s0 + s1;
          }
        }
        p[(long long)b * N + g] = v;
      }
    }
  }
}

// Node-major BF16 copy of the modes for the tensor-core expansion:
// phin[g][j] (KP = k rounded up to 16 per row, zero beyond k).
__global__ void k_phi_node_major(const __nv_bfloat16 *Phi, long long ld, int k, long long N, int KP,
                                 __nv_bfloat16 *phin) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * KP;
       e += (long long)gridDim.x * blockDim.x) {
    const long long g = e / KP;
    const int j = (int)(e % KP);
    phin[e] = j < k ? Phi[(long long)j * ld + g] : __float2bfloat16_rn(0.0f);
  }
}

// Tensor-core expansion (BF16 modes): for 128-node tiles, D = Phi_tile C with
// C = [c_1 .. c_B] (K = modes) accumulated in tensor memory, then
// p_b = mask_I (gamma_b D^-1 r_b - D[:, b] + beta_b p_b) as in k_expand_b.
// The coefficients enter as three BF16 terms (24 significant bits) staged
// once per block; the modes come from the node-major copy.  A timed-out
// completion wait writes NaN directions (reported as SDF_ERR_NONFINITE).
template <int NBP>
__global__ void __launch_bounds__(tc::GTH) k_expand_tc(const __nv_bfloat16 *__restrict__ phin,
                                                       int KP, long long N, int B,
                                                       const InstState *st, const float *cvec,
                                                       int KMAX, const uint8_t *mask,
                                                       const float *r, const float *dinv,
                                                       int dinv_per_inst, float *p) {
  using namespace tc;
  constexpr uint32_t TCOLS = NBP <= 32 ? 32 : NBP;
  extern __shared__ __align__(1024) uint8_t xsm[];
  // A: 128 nodes x KP modes; C: 3 terms x NBP instances x KP modes (64-wide K blocks)
  const int nkb = (KP + GK - 1) / GK;
  uint8_t *sa = xsm;
  uint8_t *sc = xsm + (size_t)nkb * GM * GK * 2;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  __shared__ float gam[NBP], bet[NBP];
  __shared__ int act[NBP];
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t mb = smem_u32(&mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tbase)), "r"(TCOLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(mb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int b = tid; b < NBP; b += GTH) {
    const bool on = b < B && inst_running(st[b]);
    act[b] = on ? (1 | (st[b].deflate ? 2 : 0)) : 0;
    gam[b] = on ? (float)st[b].gamma : 0.0f;
    bet[b] = on ? (float)st[b].beta : 0.0f;
  }
  __syncthreads();
  // coefficients (instances without deflation contribute zero rows)
  const size_t cterm = (size_t)nkb * NBP * GK * 2;  // bytes of one term
  for (int e = tid; e < NBP * nkb * (GK / 8); e += GTH) {
    const int b = e / (nkb * (GK / 8)), rest = e % (nkb * (GK / 8));
    const int kb = rest / (GK / 8), kg = (rest % (GK / 8)) * 8;
    __nv_bfloat16 h1[8], h2[8], h3[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int j = kb * GK + kg + i;
      const float f = ((act[b] & 2) && j < KP) ? cvec[(size_t)b * KMAX + j] : 0.0f;
      h1[i] = __float2bfloat16_rn(f);
      const float r1 = f - __bfloat162float(h1[i]);
      h2[i] = __float2bfloat16_rn(r1);
      h3[i] = __float2bfloat16_rn(r1 - __bfloat162float(h2[i]));
    }
    const size_t o = (size_t)kb * NBP * GK * 2 + cm_off(b, kg);
    *reinterpret_cast<uint4 *>(sc + o) = *reinterpret_cast<const uint4 *>(h1);
    *reinterpret_cast<uint4 *>(sc + cterm + o) = *reinterpret_cast<const uint4 *>(h2);
    *reinterpret_cast<uint4 *>(sc + 2 * cterm + o) = *reinterpret_cast<const uint4 *>(h3);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  const long long ntile = (N + GM - 1) / GM;
  bool all_ok = true;
  uint32_t phase = 0;
  for (long long t = blockIdx.x; t < ntile; t += gridDim.x) {
    const long long g0 = t * GM;
    for (int e = tid; e < GM * nkb * (GK / 8); e += GTH) {  // node rows of the modes
      const int row = e / (nkb * (GK / 8)), rest = e % (nkb * (GK / 8));
      const int kb = rest / (GK / 8), kg = (rest % (GK / 8)) * 8;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (g0 + row < N && kb * GK + kg < KP)
        val = *reinterpret_cast<const uint4 *>(phin + (g0 + row) * KP + kb * GK + kg);
      *reinterpret_cast<uint4 *>(sa + (size_t)kb * GM * GK * 2 + cm_off(row, kg)) = val;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sa), c0 = smem_u32(sc);
      const uint32_t idesc = idesc_bf16(GM, NBP);
      bool first = true;
      for (int kb = 0; kb < nkb; ++kb)
        for (int s = 0; s < GK / 16; ++s) {
          if (kb * GK + 16 * s >= KP) break;
          for (int q = 0; q < 3; ++q) {
            tc_mma(tmem, smem_desc(a0 + kb * GM * GK * 2 + s * 2 * LBO),
                   smem_desc(c0 + q * (uint32_t)cterm + kb * NBP * GK * 2 + s * 2 * LBO), idesc,
                   first ? 0u : 1u);
            first = false;
          }
        }
      tc_commit(mb);
    }
    const bool ok = mbar_wait(mb, phase, MBAR_LIMIT);
    phase ^= 1;
    tc_fence_after();
    all_ok = __syncthreads_and(ok) != 0;
    // epilogue: thread = node g (TMEM lane), columns = instances
    const long long g = g0 + warp * 32 + (tid & 31);
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    const float dsh = (!dinv_per_inst && g < N) ? dinv[g] : 0.0f;
#pragma unroll 1
    for (int cb = 0; cb < NBP; cb += 16) {
      // every load of the 16 instances first, then the arithmetic
      uint8_t mk[16];
      float rv[16], pv[16], dv[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int b = cb + q;
        const bool on = g < N && b < B && act[b];
        const long long gb = (long long)b * N + g;
        mk[q] = on ? mask[gb] : (uint8_t)1;
        rv[q] = on ? r[gb] : 0.0f;
        pv[q] = (on && bet[b] != 0.0f) ? p[gb] : 0.0f;
        dv[q] = on ? (dinv_per_inst ? dinv[gb] : dsh) : 0.0f;
      }
      float d[16];
      __syncwarp();
      if (all_ok) tc_ld16(lane_addr + (uint32_t)cb, d);
      if (g < N) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int b = cb + q;
          if (b >= B || !act[b]) continue;
          float v = 0.0f;
          if (!mk[q]) {
            v = fmaf(bet[b], pv[q], gam[b] * dv[q] * rv[q]);
            v = all_ok ? v - d[q] : __int_as_float(0x7fc00000);
          }
          p[(long long)b * N + g] = v;
        }
      }
    }
    // the next tile's MMAs overwrite the accumulator: every lane has read it
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (!all_ok) break;
  }
  if (!all_ok && tid == 0) mbar_wait(mb, phase, MBAR_LIMIT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS)
                 : "memory");
  }
}

__device__ __forceinline__ void update_epilogue(InstState &S, double rho_new, double rn2, int *cnt_slot,
                                                Ctrl *ctrl, double rtol2, int max_cg) {
  {
    *cnt_slot = 0;
    if (S.phase == 0) S.iters += 1;
    S.rnorm2 = rn2;
    const bool conv = rn2 <= rtol2 * S.bnorm2;
    if (!isfinite(rho_new) || !isfinite(rn2)) {
      S.stats.status = SDF_ERR_NONFINITE;
      S.cg_done = 1;
    } else if (S.iters >= max_cg) {
      S.stats.status = SDF_ERR_CG_MAXIT;
      S.cg_done = 1;
    } else {
      if (conv) S.await = 1;
      if (S.phase == 1) {
        S.beta = 0.0;
      } else if (S.phase == 2) {
        // Correction pass after an FP64 residual replacement: continue CG
        // (beta from the replaced iteration's rho) while the true residual is
        // close to the recurrence residual; restart (beta = 0) when the
        // recurrence had run ahead of FP32's attainable accuracy.
        S.beta = rho_new > 4.0 * S.rho ? 0.0 : rho_new / S.rho_prev;
      } else {
        S.beta = rho_new / S.rho;
      }
      if (S.phase != 2) S.rho_prev = S.rho;
      S.rho = rho_new;
      S.gamma = 1.0;
      S.csign = 1.0;
      S.phase = 0;
    }
    if (S.cg_done) {
      S.stats.cg_iters[S.outer] = S.iters;
      S.stats.relres[S.outer] = S.bnorm2 > 0 ? sqrt(rn2 / S.bnorm2) : 0.0;
      atomicSub(&ctrl->running, 1);
    }
  }
}

// Stencil part of the CG update (mixed path): x += alpha p (FP64), r -= alpha q,
// z = D^-1 r, v = S_II z - r (written for the projection GEMM), rho = (r, z),
// ||r||^2 with FP32 products summed in FP64.  The last block applies the
// convergence / beta logic of k_update (mixed = 1).
// The next direction is p = P z + Q r + beta p = z - Phi E^-1 Phi_I^T (S z - r)
// + beta p: the full A-DEF2 preconditioner P^T M^-1 + Q of the cited
// framework.  Q r vanishes in exact arithmetic (Z^T r = 0), which is why the
// FP64 path drops it; in FP32 it removes the coarse-space component that
// rounding puts into r every iteration, without which the iteration stalls.
template <int DIM>
__global__ void __launch_bounds__(NT) k_update_v(OpParams P, const double *inst, InstState *st,
                                                 const uint8_t *mask, const float *r_in,
                                                 float *r_out, const float *q, const float *p,
                                                 double *x, float *xlo, const float *dinv, float *v,
                                                 double *part, int *cnt, Ctrl *ctrl, int GX,
                                                 double rtol2, int max_cg) {
  __shared__ TileSmem<DIM, float> sm;
  __shared__ double red[NWARP];
  __shared__ int flag;
  const int b = blockIdx.x, gblk = blockIdx.y;
  InstState &S = st[b];
  if (!inst_running(S)) return;
  const long long N = P.N;
  const double alpha64 = S.alpha;
  const float alpha = (float)alpha64;
  double cb[3];
  inst_cb(P, inst + 7 * b, cb);
  const uint8_t *mk = mask + b * N;
  const float *rb = r_in + b * N, *qb = q + b * N, *pb = p + b * N;
  float *rw = r_out + b * N, *vb = v + b * N, *xl = xlo + b * N;
  double *xb = x + b * N;
  const float *db = dinv + (P.convection ? b * N : 0);
  const bool fold = S.phase == 2;  // correction pass: fold x_lo into the FP64 iterate
  KahanF rhof, rrf;
  double rho = 0.0, rr = 0.0;
  const long long T = num_tiles<DIM>(P.nx, P.ny, P.nz);
  for (long long t = gblk; t < T; t += GX) {
    int ox, oy, oz;
    tile_origin<DIM>(P, t, ox, oy, oz);
    tile_S<DIM, float>(
        P, cb, ox, oy, oz, sm,
        // r and q are zero on the active set, so z needs no mask test here
        [&](int, int, int, long long g) { return db[g] * (rb[g] - alpha * qb[g]); },
        [&](int, int, int, int, long long g, float su) {
          if (mk[g]) {
            rw[g] = 0.0f;
            vb[g] = 0.0f;
            return;
          }
          const float rn = rb[g] - alpha * qb[g];
          const float z = db[g] * rn;
          if (fold) {
            xb[g] = xb[g] + (double)xl[g] + alpha64 * (double)pb[g];
            xl[g] = 0.0f;
          } else {
            xl[g] = fmaf(alpha, pb[g], xl[g]);
          }
          rw[g] = rn;
          rhof.add(rn * z);
          rrf.add(rn * rn);
          vb[g] = su - rn;  // S z - r: the projection feeds P z + Q r (see below)
        });
  }
  rho = block_sum(rhof.value(), red);
  rr = block_sum(rrf.value(), red);
  if (threadIdx.x == 0) {
    part[((long long)b * GX + gblk) * 2 + 0] = rho;
    part[((long long)b * GX + gblk) * 2 + 1] = rr;
  }
  if (!last_block(cnt + b * NCNT + CNT_UPDATE, GX, &flag)) return;
  __shared__ double scratch[NT];
  __shared__ double tot2[2];
  reduce_fields(part + (long long)b * GX * 2, GX, 2, 2, tot2, scratch);
  if (threadIdx.x == 0) update_epilogue(S, tot2[0], tot2[1], cnt + b * NCNT + CNT_UPDATE, ctrl,
                                        rtol2, max_cg);
}

// 3D column variants (2.5D z-marching) of k_spmv and k_update_v for the mixed
// path; same arithmetic and reductions, different traversal.
// gblk: the block's slot among the GX blocks of instance b.
__device__ __forceinline__ void sigma_epilogue(InstState &S, int b, double sg, double *part, int *cnt,
                                               Ctrl *ctrl, int GX, int gblk, double *red,
                                               double *scratch, double *tot1, int *flag) {
  sg = block_sum(sg, red);
  if (threadIdx.x == 0) part[(long long)b * GX + gblk] = sg;
  if (!last_block(cnt + b * NCNT + CNT_SIGMA, GX, flag)) return;
  reduce_fields(part + (long long)b * GX, GX, 1, 1, tot1, scratch);
  if (threadIdx.x == 0) {
    double s = tot1[0];
    cnt[b * NCNT + CNT_SIGMA] = 0;
    S.sigma = s;
    if (S.phase) {
      S.alpha = 1.0;
    } else if (s > 0.0 && isfinite(s)) {
      S.alpha = S.rho / s;
    } else {
      S.stats.status = isfinite(s) ? SDF_ERR_BREAKDOWN : SDF_ERR_NONFINITE;
      S.cg_done = 1;
      S.stats.cg_iters[S.outer] = S.iters;
      atomicSub(&ctrl->running, 1);
    }
  }
}

// Column-stencil sources and outputs of the two mixed-path kernels.
struct ColSrcP {  // u = p
  static constexpr bool AUX = false;
  const float *p;
  using Raw = float;
  __device__ __forceinline__ Raw fetch(int g) const { return p[g]; }
  __device__ __forceinline__ float value(Raw r) const { return r; }
};
struct ColOutQ {  // q = S_II p (zero on the active set), sigma = (p, q)
  const uint8_t *mk;
  float *q;
  KahanF sg;
  struct Pre { uint8_t m; };
  __device__ __forceinline__ Pre fetch(int g) const { return Pre{mk[g]}; }
  __device__ __forceinline__ void store(int g, float su, float uc, float, const Pre &pr) {
    const float qv = pr.m ? 0.0f : su;
    q[g] = qv;
    sg.add(uc * qv);
  }
};
// u = z = D^-1 (r - alpha q) (r and q vanish on the active set).  (Carrying
// r - alpha q in a second shared ring for the output nodes instead of
// reloading r and q there measured slower on this part.)
struct ColSrcZ {
  static constexpr bool AUX = false;
  const float *r, *q, *dinv;
  float alpha;
  struct Raw { float r, q, d; };
  __device__ __forceinline__ Raw fetch(int g) const { return Raw{r[g], q[g], dinv[g]}; }
  __device__ __forceinline__ float aux(const Raw &a) const { return a.r - alpha * a.q; }
  __device__ __forceinline__ float value(const Raw &a) const { return a.d * aux(a); }
};
// FOLD: correction pass, which folds x_lo into the FP64 iterate.  A separate
// instantiation keeps the FP64 arithmetic (1/64 of the FP32 rate on this part)
// out of the other 99 of every 100 passes.
template <bool FOLD> struct ColOutUpd {  // r, x, v = S z - r and the CG dot products
  const uint8_t *mk;
  const float *r, *q, *p;
  float *rw, *v, *xl;
  double *x;
  float alpha;
  double alpha64;
  KahanF rho, rr;
  struct Pre { float r, q, p, xl; uint8_t m; };
  __device__ __forceinline__ Pre fetch(int g) const { return Pre{r[g], q[g], p[g], xl[g], mk[g]}; }
  __device__ __forceinline__ void store(int g, float su, float z, float, const Pre &a) {
    if (a.m) {
      rw[g] = 0.0f;
      v[g] = 0.0f;
      return;
    }
    const float rn = a.r - alpha * a.q;
    if (FOLD) {
      x[g] = x[g] + (double)a.xl + alpha64 * (double)a.p;
      xl[g] = 0.0f;
    } else {
      xl[g] = fmaf(alpha, a.p, a.xl);
    }
    rw[g] = rn;
    rho.add(rn * z);
    rr.add(rn * rn);
    v[g] = su - rn;
  }
};

template <bool VARK>
__global__ void __launch_bounds__(NT, 3) k_spmv3c(OpParams P, const double *inst, InstState *st,
                                               const uint8_t *mask, const float *p, float *q,
                                               double *part, int *cnt, Ctrl *ctrl, int GX, int zc) {
  __shared__ ColSmem<float> sm;
  __shared__ double red[NWARP], scratch[NT], tot1[1];
  __shared__ int flag;
  const int b = blockIdx.x, gblk = blockIdx.y;
  InstState &S = st[b];
  if (!inst_running(S)) return;
  const long long N = P.N;
  double cb[3];
  inst_cb(P, inst + 7 * b, cb);
  const ColSrcP src{p + b * N};
  ColOutQ out{mask + b * N, q + b * N};
  const long long items = col_items(P.nx, P.ny, P.nz, zc);
  for (long long t = gblk; t < items; t += GX) {
    int x0, y0, z0, z1;
    col_origin(P, t, zc, x0, y0, z0, z1);
    col_S3<float, VARK, false>(P, cb, x0, y0, z0, z1, sm, src, out);
  }
  sigma_epilogue(S, b, out.sg.value(), part, cnt, ctrl, GX, blockIdx.y, red, scratch, tot1, &flag);
}

template <bool VARK>
__global__ void __launch_bounds__(NT, 3) k_update_v3c(OpParams P, const double *inst, InstState *st,
                                                   const uint8_t *mask, const float *r_in,
                                                   float *r_out, const float *q, const float *p,
                                                   double *x, float *xlo, const float *dinv,
                                                   float *v, double *part, int *cnt, Ctrl *ctrl,
                                                   int GX, int zc, double rtol2, int max_cg) {
  __shared__ ColSmem<float> sm;
  __shared__ double red[NWARP], scratch[NT], tot2[2];
  __shared__ int flag;
  const int b = blockIdx.x, gblk = blockIdx.y;
  InstState &S = st[b];
  if (!inst_running(S)) return;
  const long long N = P.N;
  const double alpha64 = S.alpha;
  const float alpha = (float)alpha64;
  double cb[3];
  inst_cb(P, inst + 7 * b, cb);
  const ColSrcZ src{r_in + b * N, q + b * N, dinv + (P.convection ? b * N : 0), alpha};
  const long long items = col_items(P.nx, P.ny, P.nz, zc);
  double rho_b, rr_b;
  auto run = [&](auto out) {
    for (long long t = gblk; t < items; t += GX) {
      int x0, y0, z0, z1;
      col_origin(P, t, zc, x0, y0, z0, z1);
      col_S3<float, VARK, false>(P, cb, x0, y0, z0, z1, sm, src, out);
    }
    rho_b = out.rho.value();
    rr_b = out.rr.value();
  };
  if (S.phase == 2)
    run(ColOutUpd<true>{mask + b * N, r_in + b * N, q + b * N, p + b * N, r_out + b * N,
                        v + b * N, xlo + b * N, x + b * N, alpha, alpha64});
  else
    run(ColOutUpd<false>{mask + b * N, r_in + b * N, q + b * N, p + b * N, r_out + b * N,
                         v + b * N, xlo + b * N, x + b * N, alpha, alpha64});
  const double rho = block_sum(rho_b, red);
  const double rr = block_sum(rr_b, red);
  if (threadIdx.x == 0) {
    part[((long long)b * GX + gblk) * 2 + 0] = rho;
    part[((long long)b * GX + gblk) * 2 + 1] = rr;
  }
  if (!last_block(cnt + b * NCNT + CNT_UPDATE, GX, &flag)) return;
  reduce_fields(part + (long long)b * GX * 2, GX, 2, 2, tot2, scratch);
  if (threadIdx.x == 0) update_epilogue(S, tot2[0], tot2[1], cnt + b * NCNT + CNT_UPDATE, ctrl,
                                        rtol2, max_cg);
}

// Instance-pair variants of k_spmv3c and k_update_v3c (col_S3_pair): block x
// handles instances 2x and 2x + 1 (the second absent when B is odd).  An
// instance that is not iterating in this pass keeps every vector: its stores
// are skipped and its reduction is not entered (the half of the pair is
// computed and dropped).
struct ColSrcP2 {
  const float *p0, *p1;
  struct Raw { float a, b; };
  __device__ __forceinline__ Raw fetch(int g) const { return Raw{p0[g], p1[g]}; }
  __device__ __forceinline__ F2 value(const Raw &r) const { return F2{r.a, r.b}; }
};
struct ColOutQ2 {
  const uint8_t *m0, *m1;
  float *q0, *q1;
  bool run0, run1;
  KahanF2 sg;
  struct Pre { uint8_t a, b; };
  __device__ __forceinline__ Pre fetch(int g) const { return Pre{m0[g], m1[g]}; }
  __device__ __forceinline__ void store(int g, F2 su, F2 uc, const Pre &pr) {
    const F2 qv{pr.a ? 0.0f : su.x, pr.b ? 0.0f : su.y};
    if (run0) q0[g] = qv.x;
    if (run1) q1[g] = qv.y;
    sg.add(mul2(uc, qv));
  }
};
// u = z = D^-1 (r - alpha q) of both instances (shared D^-1: no convection)
struct ColSrcZ2 {
  const float *r0, *r1, *q0, *q1, *dinv;
  F2 nalpha;  // -alpha of each instance
  struct Raw { float r0, r1, q0, q1, d; };
  __device__ __forceinline__ Raw fetch(int g) const { return Raw{r0[g], r1[g], q0[g], q1[g], dinv[g]}; }
  __device__ __forceinline__ F2 value(const Raw &a) const {
    return mul2(bc2(a.d), fma2(nalpha, F2{a.q0, a.q1}, F2{a.r0, a.r1}));
  }
};
// FOLDANY: at least one instance is in its correction pass (folds x_lo into
// the FP64 iterate); the other 99 of every 100 passes compile without FP64 code.
template <bool FOLDANY> struct ColOutUpd2 {
  const uint8_t *m0, *m1;
  const float *r0, *r1, *q0, *q1, *p0, *p1;
  float *rw0, *rw1, *v0, *v1, *xl0, *xl1;
  double *x0, *x1;
  F2 alpha, nalpha;
  double a64_0, a64_1;
  bool run0, run1, fold0, fold1;  // fold: correction pass, x_lo folded into x
  KahanF2 rho, rr;
  struct Pre { float r0, r1, q0, q1, p0, p1, l0, l1; uint8_t m0, m1; };
  __device__ __forceinline__ Pre fetch(int g) const {
    return Pre{r0[g], r1[g], q0[g], q1[g], p0[g], p1[g], xl0[g], xl1[g], m0[g], m1[g]};
  }
  __device__ __forceinline__ void store(int g, F2 su, F2 z, const Pre &a) {
    // r, q, p and x_lo vanish on the active set, so only v needs the mask
    const F2 rn = fma2(nalpha, F2{a.q0, a.q1}, F2{a.r0, a.r1});
    F2 v = sub2(su, rn);
    if (a.m0) v.x = 0.0f;
    if (a.m1) v.y = 0.0f;
    rho.add(mul2(rn, z));
    rr.add(mul2(rn, rn));
    const F2 xn = fma2(alpha, F2{a.p0, a.p1}, F2{a.l0, a.l1});
    if (run0) {
      rw0[g] = rn.x;
      v0[g] = v.x;
      if (FOLDANY && fold0) {
        x0[g] = x0[g] + (double)a.l0 + a64_0 * (double)a.p0;
        xl0[g] = 0.0f;
      } else {
        xl0[g] = xn.x;
      }
    }
    if (run1) {
      rw1[g] = rn.y;
      v1[g] = v.y;
      if (FOLDANY && fold1) {
        x1[g] = x1[g] + (double)a.l1 + a64_1 * (double)a.p1;
        xl1[g] = 0.0f;
      } else {
        xl1[g] = xn.y;
      }
    }
  }
};

template <bool VARK>
__global__ void __launch_bounds__(NT, 3) k_spmv3p(OpParams P, InstState *st, const uint8_t *mask,
                                               const float *p, float *q, double *part, int *cnt,
                                               Ctrl *ctrl, int GX, int zc, int B) {
  __shared__ ColSmemPair sm;
  __shared__ double red[NWARP], scratch[NT], tot1[1];
  __shared__ int flag;
  const int b0 = 2 * blockIdx.y, b1 = min(b0 + 1, B - 1);
  const bool run0 = inst_running(st[b0]), run1 = b0 + 1 < B && inst_running(st[b1]);
  if (!run0 && !run1) return;
  const long long N = P.N;
  const ColSrcP2 src{p + b0 * N, p + b1 * N};
  ColOutQ2 out{mask + b0 * N, mask + b1 * N, q + b0 * N, q + b1 * N, run0, run1};
  const long long items = col_items(P.nx, P.ny, P.nz, zc);
  for (long long t = blockIdx.x; t < items; t += GX) {
    int x0, y0, z0, z1;
    col_origin(P, t, zc, x0, y0, z0, z1);
    col_S3_pair<VARK>(P, x0, y0, z0, z1, sm, src, out);
  }
  if (run0)
    sigma_epilogue(st[b0], b0, out.sg.value0(), part, cnt, ctrl, GX, blockIdx.x, red, scratch, tot1,
                   &flag);
  if (run1)
    sigma_epilogue(st[b1], b1, out.sg.value1(), part, cnt, ctrl, GX, blockIdx.x, red, scratch, tot1,
                   &flag);
}

template <bool VARK>
__global__ void __launch_bounds__(NT, 2) k_update_v3p(OpParams P, InstState *st, const uint8_t *mask,
                                                   const float *r_in, float *r_out, const float *q,
                                                   const float *p, double *x, float *xlo,
                                                   const float *dinv, float *v, double *part,
                                                   int *cnt, Ctrl *ctrl, int GX, int zc,
                                                   double rtol2, int max_cg, int B) {
  __shared__ ColSmemPair sm;
  __shared__ double red[NWARP], scratch[NT], tot2[2];
  __shared__ int flag;
  const int b0 = 2 * blockIdx.y, b1 = min(b0 + 1, B - 1);
  InstState &S0 = st[b0], &S1 = st[b1];
  const bool run0 = inst_running(S0), run1 = b0 + 1 < B && inst_running(S1);
  if (!run0 && !run1) return;
  const long long N = P.N;
  const float al0 = (float)S0.alpha, al1 = (float)S1.alpha;
  const ColSrcZ2 src{r_in + b0 * N, r_in + b1 * N, q + b0 * N, q + b1 * N, dinv, F2{-al0, -al1}};
  const bool fold0 = run0 && S0.phase == 2, fold1 = run1 && S1.phase == 2;
  const long long items = col_items(P.nx, P.ny, P.nz, zc);
  double rho[2], rr[2];
  auto run = [&](auto out) {
    for (long long t = blockIdx.x; t < items; t += GX) {
      int x0, y0, z0, z1;
      col_origin(P, t, zc, x0, y0, z0, z1);
      col_S3_pair<VARK>(P, x0, y0, z0, z1, sm, src, out);
    }
    rho[0] = out.rho.value0();
    rho[1] = out.rho.value1();
    rr[0] = out.rr.value0();
    rr[1] = out.rr.value1();
  };
#define SDF_UPD2(F_)                                                                             \
  ColOutUpd2<F_>{mask + b0 * N, mask + b1 * N, r_in + b0 * N, r_in + b1 * N, q + b0 * N,         \
                 q + b1 * N, p + b0 * N, p + b1 * N, r_out + b0 * N, r_out + b1 * N,            \
                 v + b0 * N, v + b1 * N, xlo + b0 * N, xlo + b1 * N, x + b0 * N, x + b1 * N,    \
                 F2{al0, al1}, F2{-al0, -al1}, S0.alpha, S1.alpha, run0, run1, fold0, fold1}
  if (fold0 || fold1)
    run(SDF_UPD2(true));
  else
    run(SDF_UPD2(false));
#undef SDF_UPD2
  for (int h = 0; h < 2; ++h) {
    if (!(h == 0 ? run0 : run1)) continue;
    const int b = h == 0 ? b0 : b1;
    const double rb = block_sum(rho[h], red);
    const double rrb = block_sum(rr[h], red);
    if (threadIdx.x == 0) {
      part[((long long)b * GX + blockIdx.x) * 2 + 0] = rb;
      part[((long long)b * GX + blockIdx.x) * 2 + 1] = rrb;
    }
    if (!last_block(cnt + b * NCNT + CNT_UPDATE, GX, &flag)) continue;
    reduce_fields(part + (long long)b * GX * 2, GX, 2, 2, tot2, scratch);
    if (threadIdx.x == 0)
      update_epilogue(st[b], tot2[0], tot2[1], cnt + b * NCNT + CNT_UPDATE, ctrl, rtol2, max_cg);
    __syncthreads();
  }
}

// Projection GEMM: part[gblk][b][j] = sum over block gblk's node range of
// Phi_j(g) v_b(g), for NB instances per block (NB = 1: threads split modes x
// node lanes; NB >= 16: threads split modes x instances).  FP32 products and
// chunk sums, FP64 accumulation across chunks.  v is zero on each instance's
// active set.
template <int KMAX, int NB, class PhiT>
__global__ void __launch_bounds__(NT) k_proj_gemm(const PhiT *__restrict__ Phi, long long ld, int k,
                                                  long long N, int B, const InstState *st,
                                                  const float *v, double *part, int Bpad) {
  constexpr int CH = (KMAX <= 64 && NB <= 64) ? 64 : 32;
  constexpr int MT = KMAX / 16;
  constexpr int NT_N = NB >= 16 ? NB / 16 : 1;
  __shared__ __align__(16) float Ps[CH][KMAX + 1];
  __shared__ float Vs[CH][NB + 1];
  __shared__ int run[NB];
  const int ib = blockIdx.x * NB, gblk = blockIdx.y, GXp = gridDim.y;
  for (int e = threadIdx.x; e < NB; e += NT) {
    int bb = ib + e;
    run[e] = (bb < B && !st[bb].outer_done && !st[bb].cg_done && st[bb].deflate) ? 1 : 0;
  }
  __syncthreads();
  // contiguous node range of this block, in whole chunks
  const long long nch = (N + CH - 1) / CH;
  const long long c_lo = nch * gblk / GXp, c_hi = nch * (gblk + 1) / GXp;
  const int ti = threadIdx.x / 16, tj = threadIdx.x % 16;
  KahanF acck[MT][NT_N];  // FP32 chunk sums, compensated across chunks
  for (long long ch = c_lo; ch < c_hi; ++ch) {
    const long long g0 = ch * CH;
    for (int e = threadIdx.x; e < CH * KMAX; e += NT) {
      int c = e % CH, j = e / CH;
      long long g = g0 + c;
      Ps[c][j] = (j < k && g < N) ? (float)Phi[(long long)j * ld + g] : 0.0f;
    }
    for (int e = threadIdx.x; e < CH * NB; e += NT) {
      int c = e % CH, bq = e / CH;
      long long g = g0 + c;
      Vs[c][bq] = (run[bq] && g < N) ? v[(long long)(ib + bq) * N + g] : 0.0f;
    }
    __syncthreads();
    float acc[MT][NT_N];
#pragma unroll
    for (int a = 0; a < MT; ++a)
#pragma unroll
      for (int c = 0; c < NT_N; ++c) acc[a][c] = 0.0f;
    if constexpr (NB >= 16) {
#pragma unroll 8
      for (int c = 0; c < CH; ++c) {
        float pa[MT], vb[NT_N];
#pragma unroll
        for (int a = 0; a < MT; ++a) pa[a] = Ps[c][ti + 16 * a];
#pragma unroll
        for (int q = 0; q < NT_N; ++q) vb[q] = Vs[c][tj + 16 * q];
#pragma unroll
        for (int a = 0; a < MT; ++a)
#pragma unroll
          for (int q = 0; q < NT_N; ++q) acc[a][q] = fmaf(pa[a], vb[q], acc[a][q]);
      }
    } else {  // NB == 1: lane tj takes nodes tj, tj + 16, ... of the chunk
#pragma unroll
      for (int c = tj; c < CH; c += 16) {
        const float vv = Vs[c][0];
#pragma unroll
        for (int a = 0; a < MT; ++a) acc[a][0] = fmaf(Ps[c][ti + 16 * a], vv, acc[a][0]);
      }
    }
#pragma unroll
    for (int a = 0; a < MT; ++a)
#pragma unroll
      for (int q = 0; q < NT_N; ++q) acck[a][q].add(acc[a][q]);
    __syncthreads();
  }
  if constexpr (NB >= 16) {
#pragma unroll
    for (int a = 0; a < MT; ++a)
#pragma unroll
      for (int q = 0; q < NT_N; ++q) {
        int j = ti + 16 * a, bb = ib + tj + 16 * q;
        if (bb < Bpad) part[((long long)gblk * Bpad + bb) * KMAX + j] = acck[a][q].value();
      }
  } else {  // reduce the 16 node lanes through shared memory (reuse Ps)
    double *red = reinterpret_cast<double *>(&Ps[0][0]);  // KMAX*16 doubles fit in Ps
#pragma unroll
    for (int a = 0; a < MT; ++a) red[(ti + 16 * a) * 16 + tj] = acck[a][0].value();
    __syncthreads();
    for (int j = threadIdx.x; j < KMAX; j += NT) {
      double sum = 0.0;
      for (int l = 0; l < 16; ++l) sum += red[j * 16 + l];
      part[((long long)gblk * Bpad + ib) * KMAX + j] = sum;
    }
  }
}

// Tensor-core projection (BF16 modes): part[blk][b][j] = sum over block blk's
// node range of Phi_j(g) v_b(g), for every instance of the batch at once.
// D (modes x instances) accumulates in tensor memory over the block's 64-node
// chunks; A = the modes' rows (K = nodes, contiguous in the column-major Phi),
// B = the instances' rows of v (K = nodes, contiguous).  v is FP32: it enters
// as three BF16 terms v1 = bf16(v), v2 = bf16(v - v1), v3 = bf16(v - v1 - v2)
// (24 significant bits), each multiplied by the exactly stored modes.  A
// timed-out completion wait leaves NaN partials, which the CG reports as
// SDF_ERR_NONFINITE.
template <int NBP>
__global__ void __launch_bounds__(tc::GTH) k_proj_tc(const __nv_bfloat16 *__restrict__ Phi,
                                                     long long ld, int k, long long N, int B,
                                                     const InstState *st, const float *v,
                                                     double *part, int Bpad, int KM) {
  using namespace tc;
  static_assert(NBP % 16 == 0 && NBP >= 16 && NBP <= 256, "batch tile");
  constexpr uint32_t TCOLS = NBP <= 32 ? 32 : NBP;
  extern __shared__ __align__(1024) uint8_t tsm[];
  uint8_t *sa = tsm;              // 128 modes x 64 nodes (rows >= k zero)
  uint8_t *sb = tsm + GM * GK * 2;  // 3 terms x NBP instances x 64 nodes
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  __shared__ int run[NBP];
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t mb = smem_u32(&mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tbase)), "r"(TCOLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(mb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int b = tid; b < NBP; b += GTH)
    run[b] = (b < B && !st[b].outer_done && !st[b].cg_done && st[b].deflate) ? 1 : 0;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  const long long nch = (N + GK - 1) / GK;
  const long long c_lo = nch * blockIdx.x / gridDim.x, c_hi = nch * (blockIdx.x + 1) / gridDim.x;
  const bool vphi = (ld % 8) == 0, vv = (N % 4) == 0;
  // The next chunk's global loads are issued into registers before this
  // chunk's MMAs are awaited (the instance rows too when NBP <= 64).
  // only the k real mode rows are staged per chunk; rows k..127 are zeroed once
  constexpr int AIT = GM * (GK / 8) / GTH, BIT = NBP * (GK / 8) / GTH;
  const int a_items = k * (GK / 8);
  for (int e = a_items + tid; e < GM * (GK / 8); e += GTH)
    *reinterpret_cast<uint4 *>(sa + cm_off(e >> 3, (e & 7) * 8)) = make_uint4(0, 0, 0, 0);
  constexpr bool PFB = NBP <= 64;
  uint4 pa[AIT];
  float pb[PFB ? BIT : 1][8];
  auto fetch_a = [&](long long ch) {
    const long long g0 = ch * GK;
#pragma unroll
    for (int it = 0; it < AIT; ++it) {
      const int e = tid + it * GTH, j = e >> 3, kg = (e & 7) * 8;
      const long long g = g0 + kg;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (e < a_items && g < N) {
        const __nv_bfloat16 *src = Phi + (long long)j * ld + g;
        if (vphi && g + 8 <= N) {
          val = *reinterpret_cast<const uint4 *>(src);
        } else {
          __nv_bfloat16 h[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) h[q] = g + q < N ? src[q] : __float2bfloat16_rn(0.0f);
          val = *reinterpret_cast<const uint4 *>(h);
        }
      }
      pa[it] = val;
    }
  };
  auto fetch_b = [&](long long ch, int it, float (&f)[8]) {
    const int e = tid + it * GTH, b = e >> 3, kg = (e & 7) * 8;
    const long long g = ch * GK + kg;
#pragma unroll
    for (int q = 0; q < 8; ++q) f[q] = 0.0f;
    if (run[b] && g < N) {
      const float *src = v + (long long)b * N + g;
      if (vv && g + 8 <= N) {
        const float4 a = *reinterpret_cast<const float4 *>(src);
        const float4 c = *reinterpret_cast<const float4 *>(src + 4);
        f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w;
        f[4] = c.x; f[5] = c.y; f[6] = c.z; f[7] = c.w;
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) f[q] = g + q < N ? src[q] : 0.0f;
      }
    }
  };
  auto put_b = [&](int it, const float (&f)[8]) {  // three BF16 terms of 8 values
    const int e = tid + it * GTH, b = e >> 3, kg = (e & 7) * 8;
    __nv_bfloat16 h1[8], h2[8], h3[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      h1[q] = __float2bfloat16_rn(f[q]);
      const float r1 = f[q] - __bfloat162float(h1[q]);
      h2[q] = __float2bfloat16_rn(r1);
      h3[q] = __float2bfloat16_rn(r1 - __bfloat162float(h2[q]));
    }
    const uint32_t o = cm_off(b, kg);
    *reinterpret_cast<uint4 *>(sb + o) = *reinterpret_cast<const uint4 *>(h1);
    *reinterpret_cast<uint4 *>(sb + NBP * 128 + o) = *reinterpret_cast<const uint4 *>(h2);
    *reinterpret_cast<uint4 *>(sb + 2 * NBP * 128 + o) = *reinterpret_cast<const uint4 *>(h3);
  };
  if (c_lo < c_hi) {
    fetch_a(c_lo);
    if constexpr (PFB) {
#pragma unroll
      for (int it = 0; it < BIT; ++it) fetch_b(c_lo, it, pb[it]);
    }
  }
  bool all_ok = true;
  uint32_t phase = 0;
  for (long long ch = c_lo; ch < c_hi; ++ch) {
    // the tiles are free: the previous chunk's MMAs have completed
#pragma unroll
    for (int it = 0; it < AIT; ++it) {
      const int e = tid + it * GTH;
      if (e < a_items) *reinterpret_cast<uint4 *>(sa + cm_off(e >> 3, (e & 7) * 8)) = pa[it];
    }
    if constexpr (PFB) {
#pragma unroll
      for (int it = 0; it < BIT; ++it) put_b(it, pb[it]);
    } else {
      for (int it = 0; it < BIT; ++it) {
        float f[8];
        fetch_b(ch, it, f);
        put_b(it, f);
      }
    }
    if (ch + 1 < c_hi) {
      fetch_a(ch + 1);
      if constexpr (PFB) {
#pragma unroll
        for (int it = 0; it < BIT; ++it) fetch_b(ch + 1, it, pb[it]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
      const uint32_t idesc = idesc_bf16(GM, NBP);
#pragma unroll
      for (int s = 0; s < GK / 16; ++s)
#pragma unroll
        for (int t = 0; t < 3; ++t)
          tc_mma(tmem, smem_desc(a0 + s * 2 * LBO), smem_desc(b0 + t * NBP * 128 + s * 2 * LBO),
                 idesc, (ch > c_lo || s > 0 || t > 0) ? 1u : 0u);
      tc_commit(mb);
    }
    const bool ok = mbar_wait(mb, phase, MBAR_LIMIT);
    phase ^= 1;
    tc_fence_after();
    all_ok = __syncthreads_and(ok) != 0;
    if (!all_ok) break;
  }
  // epilogue: lane j of warp w (row 32 w + j) holds mode 32 w + j
  const int j = warp * 32 + (tid & 31);
  const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
  const bool any = c_hi > c_lo;
#pragma unroll 1
  for (int c0 = 0; c0 < NBP; c0 += 16) {
    float d[16];
    __syncwarp();
    if (any && all_ok) tc_ld16(lane_addr + (uint32_t)c0, d);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int b = c0 + q;
      if (j < KM && b < Bpad) {
        const double val = !all_ok ? __longlong_as_double(0x7ff8000000000000LL)
                                   : (any ? (double)d[q] : 0.0);
        part[((long long)blockIdx.x * Bpad + b) * KM + j] = val;
      }
    }
  }
  if (!all_ok && tid == 0) mbar_wait(mb, phase, MBAR_LIMIT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS)
                 : "memory");
  }
}

// Sum the projection partials of each instance in block order and form the
// coarse coefficients c_b = csign_b E_raw,b^-1 t_b (FP64), stored as FP32.
template <int KMAX, class CT = float>
__global__ void __launch_bounds__(NT) k_proj_reduce(const double *part, int GXp, int Bpad, int k,
                                                    const InstState *st, const double *Einv,
                                                    CT *cvec) {
  // NT threads: mode j = tid % KMAX, block slice q = tid / KMAX sums the
  // partials g = q, q + Q, ... (eight loads in flight), then the Q slice sums
  // of each mode are added in slice order (deterministic)
  constexpr int Q = NT / KMAX > 0 ? NT / KMAX : 1;
  __shared__ double t[KMAX];
  __shared__ double sl[Q][KMAX];
  const int b = blockIdx.x;
  const InstState &S = st[b];
  if (S.outer_done || S.cg_done) return;
  for (int e = threadIdx.x; e < Q * KMAX; e += blockDim.x) {
    const int j = e % KMAX, q = e / KMAX;
    double s = 0.0;
    if (j < k && S.deflate) {
#pragma unroll 8
      for (int g = q; g < GXp; g += Q) s += part[((long long)g * Bpad + b) * KMAX + j];
    }
    sl[q][j] = s;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < KMAX; j += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < Q; ++q) s += sl[q][j];
    t[j] = s;
  }
  __syncthreads();
  const double *Ei = Einv + (size_t)b * k * k;
  for (int i = threadIdx.x; i < KMAX; i += blockDim.x) {
    double c = 0.0;
    if (i < k && S.deflate) {
      for (int j = 0; j < k; ++j) c = fma(Ei[i * k + j], t[j], c);
      c *= S.csign;
    }
    cvec[(size_t)b * KMAX + i] = (CT)c;
  }
}

// ---------------------------------------------------------------------------
// FP64 path, shared-Phi batch kernels (batches of kFp64BatchMin instances or
// more): the projection t_b = Phi_I^T v_b of every instance is one
// tall-skinny GEMM over shared-memory chunks, each mode row read once per tile
// of NB instances; the expansion p_b = gamma_b D^-1 r_b + beta_b p_b - Phi c_b
// reads each node's mode values once per group of IG instances.  The
// arithmetic is the per-instance kernels' (FP64 products and sums, c_b =
// csign E_raw^-1 t_b from k_proj_reduce); only the order of the partial sums
// differs.  On this part the FP64 pipe (about 2 FMA per clock per SM) binds
// these kernels: sharing Phi cuts its reads from 2k to 2k / (tile) doubles per
// node and instance, the FMA count (k each) stays.
constexpr int kFp64BatchMin = 8;
constexpr int kExpandGroup = 32;

template <int KMAX, int NB>
__global__ void __launch_bounds__(NT) k_proj_gemm64(const double *__restrict__ Phi, long long ld,
                                                    int k, long long N, int B, const InstState *st,
                                                    const double *__restrict__ v, double *part,
                                                    int Bpad) {
  static_assert(NB >= 16 && NB % 16 == 0 && KMAX % 16 == 0, "thread tile");
  constexpr int CH = (KMAX * NB >= 128 * 64) ? 16 : 32;
  constexpr int MT = KMAX / 16, NTN = NB / 16;
  __shared__ double Ps[CH][KMAX + 1];
  __shared__ double Vs[CH][NB + 1];
  __shared__ int run[NB];
  const int ib = blockIdx.x * NB, gblk = blockIdx.y, GXp = gridDim.y;
  for (int e = threadIdx.x; e < NB; e += NT) {
    const int bb = ib + e;
    run[e] = (bb < B && !st[bb].outer_done && !st[bb].cg_done && st[bb].deflate) ? 1 : 0;
  }
  __syncthreads();
  const long long nch = (N + CH - 1) / CH;
  const long long c_lo = nch * gblk / GXp, c_hi = nch * (gblk + 1) / GXp;
  const int ti = threadIdx.x / 16, tj = threadIdx.x % 16;
  double acc[MT][NTN];
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int q = 0; q < NTN; ++q) acc[a][q] = 0.0;
  for (long long ch = c_lo; ch < c_hi; ++ch) {
    const long long g0 = ch * CH;
    for (int e = threadIdx.x; e < CH * KMAX; e += NT) {
      const int c = e % CH, j = e / CH;
      const long long g = g0 + c;
      Ps[c][j] = (j < k && g < N) ? Phi[(long long)j * ld + g] : 0.0;
    }
    for (int e = threadIdx.x; e < CH * NB; e += NT) {
      const int c = e % CH, q = e / CH;
      const long long g = g0 + c;
      Vs[c][q] = (run[q] && g < N) ? v[(long long)(ib + q) * N + g] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < CH; ++c) {
      double pa[MT], vb[NTN];
#pragma unroll
      for (int a = 0; a < MT; ++a) pa[a] = Ps[c][ti + 16 * a];
#pragma unroll
      for (int q = 0; q < NTN; ++q) vb[q] = Vs[c][tj + 16 * q];
#pragma unroll
      for (int a = 0; a < MT; ++a)
#pragma unroll
        for (int q = 0; q < NTN; ++q) acc[a][q] = fma(pa[a], vb[q], acc[a][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int q = 0; q < NTN; ++q) {
      const int j = ti + 16 * a, bb = ib + tj + 16 * q;
      if (bb < Bpad) part[((long long)gblk * Bpad + bb) * KMAX + j] = acc[a][q];
    }
}

// Grid: x = instance group of IG (fastest, so that the groups of one node
// range run together and share its mode rows in L2), y = node range.
template <int KMAX, int IG>
__global__ void __launch_bounds__(NT) k_expand64_b(const double *__restrict__ Phi, long long ld,
                                                   int k, long long N, int B, const InstState *st,
                                                   const double *cvec, const uint8_t *mask,
                                                   const double *r, const double *dinv,
                                                   int dinv_per_inst, double *p) {
  __shared__ double cs[KMAX][IG];  // coefficients, mode-major: a warp reads one broadcast value
  __shared__ double gam[IG], bet[IG];
  __shared__ int act[IG];
  const int b0 = blockIdx.x * IG;
  for (int q = threadIdx.x; q < IG; q += NT) {
    const int b = b0 + q;
    const bool on = b < B && inst_running(st[b]);
    act[q] = on ? (1 | (st[b].deflate ? 2 : 0)) : 0;
    gam[q] = on ? st[b].gamma : 0.0;
    bet[q] = on ? st[b].beta : 0.0;
  }
  for (int e = threadIdx.x; e < IG * KMAX; e += NT) {
    const int q = e / KMAX, j = e % KMAX;
    cs[j][q] = (b0 + q < B) ? cvec[(size_t)(b0 + q) * KMAX + j] : 0.0;
  }
  __syncthreads();
  bool any = false;
  for (int q = 0; q < IG; ++q) any = any || act[q];
  if (!any) return;
  // sub-groups of 8 instances: 8 accumulators per thread; a node's mode
  // values are re-read per sub-group from L1
  constexpr int SG = 8;
  static_assert(IG % SG == 0, "sub-groups");
  for (long long g = (long long)blockIdx.y * NT + threadIdx.x; g < N;
       g += (long long)gridDim.y * NT) {
    const double d_shared = dinv_per_inst ? 0.0 : dinv[g];
#pragma unroll 1
    for (int q0 = 0; q0 < IG; q0 += SG) {
      int on = 0, dfl = 0;
#pragma unroll
      for (int u = 0; u < SG; ++u) {
        on |= act[q0 + u];
        dfl |= act[q0 + u] & 2;
      }
      if (!on) continue;  // uniform across the block
      double acc[SG];
#pragma unroll
      for (int u = 0; u < SG; ++u) acc[u] = 0.0;
      if (dfl) {
        for (int j = 0; j < k; ++j) {
          const double ph = Phi[(long long)j * ld + g];
#pragma unroll
          for (int u = 0; u < SG; ++u) acc[u] = fma(ph, cs[j][q0 + u], acc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < SG; ++u) {
        const int q = q0 + u;
        if (!act[q]) continue;
        const long long gb = (long long)(b0 + q) * N + g;
        double val = 0.0;
        if (!mask[gb]) {
          const double dv = dinv_per_inst ? dinv[gb] : d_shared;
          val = gam[q] * dv * r[gb];
          if (bet[q] != 0.0) val = fma(bet[q], p[gb], val);
          if (act[q] & 2) val -= acc[u];
        }
        p[gb] = val;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Active-set update (App. B.1 lines 7-11): y = psi on A, x on I;
// A_new = {y > psi - tau}; count changes; stop when A_new = A.
__global__ void __launch_bounds__(NT) k_active(long long N, const double *psi, uint8_t *mask,
                                               const double *x, const float *xlo, double *y,
                                               InstState *st, double *part, int *cnt, Ctrl *ctrl,
                                               int GX, double tau, int max_outer) {
  __shared__ double red[NWARP];
  __shared__ int flag;
  const int b = blockIdx.x, gblk = blockIdx.y;
  InstState &S = st[b];
  if (S.outer_done) return;
  const bool failed = S.stats.status != SDF_OK;
  uint8_t *mk = mask + b * N;
  const double *xb = x + b * N;
  double *yb = y + b * N;
  double ch = 0.0;
  for (long long g = (long long)gblk * NT + threadIdx.x; g < N; g += (long long)GX * NT) {
    uint8_t a = mk[g];
    double yv = a ? psi[g] : (xlo ? xb[g] + (double)xlo[b * N + g] : xb[g]);
    yb[g] = yv;
    if (!failed) {
      uint8_t an = yv > psi[g] - tau ? 1 : 0;
      if (an != a) {
        ch += 1.0;
        mk[g] = an;
      }
    }
  }
  ch = block_sum(ch, red);
  if (threadIdx.x == 0) part[b * GX + gblk] = ch;
  if (!last_block(cnt + b * NCNT + CNT_ACTIVE, GX, &flag)) return;
  __shared__ double scratch[NT];
  __shared__ double tot1[1];
  reduce_fields(part + (long long)b * GX, GX, 1, 1, tot1, scratch);
  if (threadIdx.x == 0) {
    double s = tot1[0];
    cnt[b * NCNT + CNT_ACTIVE] = 0;
    S.changes = (int)s;
    S.stats.outer_iters = S.outer + 1;
    if (failed) {
      S.outer_done = 1;
    } else if (S.changes == 0) {
      S.outer_done = 1;
    } else if (S.outer + 1 >= max_outer) {
      S.outer_done = 1;
      S.stats.status = SDF_ERR_OUTER_MAXIT;
    } else {
      S.outer += 1;
      atomicAdd(&ctrl->live, 1);
    }
  }
}

// lambda = rhs - S y on the whole grid (Eq. schur).
template <int DIM>
__global__ void __launch_bounds__(NT) k_lambda(OpParams P, const double *inst, const double *y,
                                               double *lam, int GX) {
  __shared__ TileSmem<DIM> sm;
  const int b = blockIdx.x, gblk = blockIdx.y;
  const long long N = P.N;
  const double *ib = inst + 7 * b;
  double cb[3];
  inst_cb(P, ib, cb);
  const double *yb = y + b * N;
  double *lb = lam + b * N;
  const long long T = num_tiles<DIM>(P.nx, P.ny, P.nz);
  for (long long t = gblk; t < T; t += GX) {
    int ox, oy, oz;
    tile_origin<DIM>(P, t, ox, oy, oz);
    tile_S<DIM>(
        P, cb, ox, oy, oz, sm, [&](int, int, int, long long g) { return yb[g]; },
        [&](int, int gx, int gy, int gz, long long g, double su) {
          lb[g] = (P.rhs ? P.rhs[b * N + g] : P.mass * desired(P, ib, gx, gy, gz)) - su;
        });
  }
}

// sdf_apply_S building block: out = S_II u (mode 0) or S u (mode 1), for
// column blockIdx.y of u and out (column stride P.N; one column from the ABI,
// a whole block from the restricted eigensolve).
template <int DIM>
__global__ void __launch_bounds__(NT) k_apply(OpParams P, const double *inst,
                                              const uint8_t *mask, const double *u, double *out,
                                              int mode, int GX) {
  __shared__ TileSmem<DIM> sm;
  double cb[3];
  inst_cb(P, inst, cb);
  u += (long long)blockIdx.y * P.N;
  out += (long long)blockIdx.y * P.N;
  const long long T = num_tiles<DIM>(P.nx, P.ny, P.nz);
  for (long long t = blockIdx.x; t < T; t += GX) {
    int ox, oy, oz;
    tile_origin<DIM>(P, t, ox, oy, oz);
    tile_S<DIM>(
        P, cb, ox, oy, oz, sm,
        [&](int, int, int, long long g) { return (mode == 0 && mask[g]) ? 0.0 : u[g]; },
        [&](int, int, int, int, long long g, double su) {
          out[g] = (mode == 0 && mask[g]) ? 0.0 : su;
        });
  }
}

// Space-time Kronecker basis (App. E.2.1 Eq. kron_basis): column
// c = l r + j of Phi (N rows, leading dimension ld) is spatial mode j
// (zs, Ns rows, leading dimension ldz) on time step l, zero elsewhere.
template <class T>
__global__ void k_kron_time(const T *zs, long long ldz, int r, long long Ns, int nt, T *phi,
                            long long ld) {
  const long long N = Ns * nt, total = N * (long long)r * nt;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / N, g = e - c * N;
    const int l = (int)(c / r), j = (int)(c - (long long)l * r);
    const long long slab = g / Ns;
    phi[c * ld + g] = slab == l ? zs[j * ldz + (g - slab * Ns)] : T(0.0f);
  }
}

// Space-time basis W_t (x) Z_s (App. E.2.1): column c = a r + j of Phi is
// spatial mode j times W_t[l, a] on time step l.  W_t (n_t x r_t,
// column-major) travels in the kernel's parameters.
constexpr int SDF_TB_MAX = 1024;
struct TemporalBasis {
  int nt, rt;
  double w[SDF_TB_MAX];
};
template <class T>
__global__ void k_time_basis(const TemporalBasis tb, const T *zs, long long ldz, int r, long long Ns,
                             T *phi, long long ld) {
  const long long N = Ns * tb.nt, total = N * (long long)r * tb.rt;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / N, g = e - c * N;
    const int a = (int)(c / r), j = (int)(c - (long long)a * r);
    const int l = (int)(g / Ns);
    const double v = tb.w[l + a * tb.nt] * (double)zs[j * ldz + (g - (long long)l * Ns)];
    phi[c * ld + g] = (T)v;
  }
}

// Kronecker sine modes (Sec. 2.2.8): Phi_c(j) = prod_l sqrt(2/(n_l+1)) sin(i_l pi j_l/(n_l+1)).
struct ModeIdx {
  int v[3 * SDF_MAX_K];
};

template <class PhiT>
__global__ void k_sine_modes(int dim, int nx, int ny, int nz, ModeIdx idx, int k, PhiT *Phi,
                             long long ld) {
  long long N = (long long)nx * ny * nz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * k;
       e += (long long)gridDim.x * blockDim.x) {
    int c = (int)(e / N);
    long long g = e % N;
    int j0 = (int)(g % nx);
    long long t = g / nx;
    int j1 = (int)(t % ny), j2 = (int)(t / ny);
    double v = sqrt(2.0 / (nx + 1)) * sinpi((double)idx.v[3 * c] * (j0 + 1) / (nx + 1));
    v *= sqrt(2.0 / (ny + 1)) * sinpi((double)idx.v[3 * c + 1] * (j1 + 1) / (ny + 1));
    if (dim == 3) v *= sqrt(2.0 / (nz + 1)) * sinpi((double)idx.v[3 * c + 2] * (j2 + 1) / (nz + 1));
    Phi[(long long)c * ld + g] = (PhiT)v;
  }
}

}  // namespace

// ===========================================================================
// host side

struct sdf_problem {
  sdf_problem_desc d;
  std::vector<double> kappa;
  OpParams P;
  bool bound = false;
  int device = -1;  // CUDA device current when the problem buffer was bound
  void *dev = nullptr;
  size_t dev_bytes = 0;
  double *dinv_shared = nullptr;
  float *dinv_shared32 = nullptr;
  const void *phi = nullptr;
  int k = 0;
  long long ld = 0;
  sdf_dtype phi_dtype = SDF_F64;
  std::string err;
  int nsm = 148;
  int *pinned = nullptr;  // 2 ints of pinned host memory for polling
  sdf_profile prof{};
  cudaEvent_t ev[8] = {};
  bool ev_ready = false;
  const double *x0 = nullptr;  // start of every inner solve (set for one call)
  // autotuned column depth of the 3D mixed kernels, keyed by batch size
  std::map<int, int> tuned_zc;
  std::map<int, int> tuned_pairs;  // 1: instance pairs, 0: one instance per block
  cudaStream_t cap_stream = nullptr;  // private stream the CG chunks are captured on
  int force_zc = 0;     // set by sdf_autotune while it times one candidate
  int force_pairs = 0;  // the same for the pairing (1 pairs, 2 single)
  // a problem created from its operator K (sdf_problem_create_csr): the
  // assembled S = mass I + wgt K^T K and its inverse diagonal, host copies
  bool csr = false;
  std::vector<int> srp, sci;
  std::vector<double> sv, sdinv;
};

namespace {

sdf_status fail(sdf_problem *p, sdf_status s, const std::string &msg) {
  if (p) p->err = msg;
  return s;
}

sdf_status cuda_check(sdf_problem *p, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return SDF_OK;
  return fail(p, SDF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                               \
  do {                                                         \
    sdf_status _s = cuda_check(p, (call), #call);              \
    if (_s != SDF_OK) return _s;                               \
  } while (0)
#define CKL(what)                                              \
  do {                                                         \
    sdf_status _s = cuda_check(p, cudaGetLastError(), what);   \
    if (_s != SDF_OK) return _s;                               \
  } while (0)

int kmax_for(int k) { return k <= 16 ? 16 : k <= 32 ? 32 : k <= 64 ? 64 : 128; }

Layout make_layout(const sdf_problem *p, int B, int max_blocks = 0, int mixed = 0,
                   int column_depth = 0, int column_pairs = 0) {
  Layout L{};
  const long long N = p->P.N;
  const int k = std::max(p->k, 1), KM = kmax_for(k);
  long long T = p->d.dim == 1   ? num_tiles<1>(p->P.nx, p->P.ny, p->P.nz)
                : p->d.dim == 2 ? num_tiles<2>(p->P.nx, p->P.ny, p->P.nz)
                                : num_tiles<3>(p->P.nx, p->P.ny, p->P.nz);
  // FP64 path: two blocks per SM in total (FP64-pipe bound, large partials);
  // mixed path: eight (latency-bound stencil tiles need more resident blocks)
  long long target = (long long)p->nsm * (mixed ? 8 : 2);
  L.gx = (int)std::max<long long>(1, std::min<long long>(T, (target + B - 1) / B));
  long long chunks = (N + NT - 1) / NT;
  L.gxa = (int)std::max<long long>(1, std::min<long long>(chunks, (p->nsm * 8LL + B - 1) / B));
  L.gxg = (int)std::max<long long>(1, std::min<long long>((N + 15) / 16, p->nsm * 2LL));
  if (max_blocks > 0) {
    L.gx = std::min(L.gx, max_blocks);
    L.gxa = std::min(L.gxa, max_blocks);
  }
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = al(o + bytes);
    return at;
  };
  size_t vec = sizeof(double) * (size_t)N * B;
  size_t vecv = (mixed ? sizeof(float) : sizeof(double)) * (size_t)N * B;
  L.x = take(vec);
  L.b64 = take(vec);
  L.r = take(vecv);
  L.r2 = take(vecv);
  L.p = take(vecv);
  L.q = take(vecv);
  L.w = take(mixed ? vecv : 8);
  L.dinv = take(p->P.convection ? vecv : 8);
  L.mask = take((size_t)N * B);
  L.W = take(sizeof(double) * (size_t)N * k);
  size_t kk = sizeof(double) * (size_t)k * k;
  L.Einv = take(kk * B);
  L.Eraw = take(kk * B);
  L.G = take(kk * B);
  L.coarse = take(kk * B * 5);
  // 3D column traversal of the mixed path: z-chunks of zc planes (an
  // autotuned depth when sdf_autotune has measured this batch size)
  L.zc = B >= 8 ? 32 : (B >= 2 ? 16 : 8);
  {
    auto it = p->tuned_zc.find(B);
    if (it != p->tuned_zc.end()) L.zc = it->second;
    if (p->force_zc > 0) L.zc = p->force_zc;
    if (column_depth > 0) L.zc = column_depth;
    L.pairs = B >= 2 ? 1 : 0;
    auto ip = p->tuned_pairs.find(B);
    if (ip != p->tuned_pairs.end()) L.pairs = ip->second;
    const int fp = p->force_pairs > 0 ? p->force_pairs : column_pairs;
    if (fp == 1) L.pairs = B >= 2 ? 1 : 0;
    if (fp == 2) L.pairs = 0;
  }
  L.gxc = 1;
  int gxc_max = 1;  // the partial buffers fit every candidate depth (8 planes)
  if (p->d.dim == 3) {
    long long items = col_items(p->P.nx, p->P.ny, p->P.nz, L.zc);
    // one column item per block: the hardware block scheduler balances the
    // items of all instances across the SMs
    L.gxc = (int)std::max<long long>(1, std::min<long long>(items, 65535));
    if (max_blocks > 0) L.gxc = std::min(L.gxc, max_blocks);
    gxc_max = (int)std::max<long long>(
        1, std::min<long long>(col_items(p->P.nx, p->P.ny, p->P.nz, 8), 65535));
    gxc_max = std::max(gxc_max, L.gxc);
  }
  int gmax = std::max(std::max(L.gx, gxc_max), std::max(L.gxa, 1));
  L.part = take(sizeof(double) * (size_t)B * gmax * (KM + 4));
  L.gpart = take(sizeof(double) * (size_t)L.gxg * k * k);
  L.state = take(sizeof(InstState) * (size_t)B);
  L.cnt = take(sizeof(int) * (size_t)B * NCNT);
  L.ctrl = take(sizeof(Ctrl));
  // mixed path: v = S_II z, coarse coefficients, projection-GEMM partials
  L.nb = B == 1 ? 1 : (B <= 16 ? 16 : (B <= 32 ? 32 : 64));
  L.bpad = (int)(((B + L.nb - 1) / L.nb) * L.nb);
  L.gxp = std::max(1, (p->nsm * 6) / ((B + L.nb - 1) / L.nb));
  // BF16 modes: the projection runs on the tensor cores for the whole batch
  L.tcp = (mixed && p->phi_dtype == SDF_BF16 && B <= 256) ? 1 : 0;
  L.nbp = B <= 16 ? 16 : (B <= 32 ? 32 : (B <= 64 ? 64 : (B <= 128 ? 128 : 256)));
  if (L.tcp) {
    // one wave: as many blocks per SM as shared memory admits (at most 6)
    // (the 64-wide tile holds its prefetched rows in 128 registers: 4 blocks)
    const int occ = std::max(1, std::min(L.nbp == 64 ? 4 : 6,
                                         (int)((220 * 1024) / (16384 + 3 * 128 * L.nbp + 2048))));
    L.bpad = L.nbp;
    L.gxp = (int)std::min<long long>((long long)p->nsm * occ, (N + 63) / 64);
  }
  if (max_blocks > 0) L.gxp = std::min(L.gxp, max_blocks);
  L.fb = (!mixed && B >= kFp64BatchMin && p->k > 0) ? 1 : 0;
  L.v = take(mixed ? sizeof(float) * (size_t)N * B : (L.fb ? sizeof(double) * (size_t)N * B : 8));
  L.xlo = take(mixed ? sizeof(float) * (size_t)N * B : 8);
  L.cvec = take((L.fb ? sizeof(double) : sizeof(float)) * (size_t)B * KM);
  L.ppart = take((mixed || L.fb) ? sizeof(double) * (size_t)L.gxp * L.bpad * KM : 8);
  // tensor-core expansion: BF16 modes, and its shared-memory tiles must fit
  L.kp = (std::max(k, 1) + 15) / 16 * 16;
  L.tce = (L.tcp && expand_tc_smem(L.nbp, L.kp) <= 200 * 1024) ? 1 : 0;
  L.phin = take(L.tce ? sizeof(uint16_t) * (size_t)N * L.kp : 8);
  L.total = o;
  return L;
}

bool aligned(const void *ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

template <class PhiT>
const PhiT *phi_as(const sdf_problem *p) { return static_cast<const PhiT *>(p->phi); }

// The solve, templated on dimension, mode-count bucket, Phi type and vector
// precision V (double: FP64 path; float: mixed path with FP64 x, b,
// reductions, coarse operator and periodic FP64 residual replacement).
// Conditioning-based safe merge (Sec. 2.2.5, Algorithm safe) after k_coarse,
// in the coordinates of the registered pool [eigenmodes (first r) | POD
// candidates]: a basis column is a coefficient vector t with Z = Phi_I t, so
// inner products are t^T G t (G = Phi_I^T Phi_I) and the Galerkin matrix is
// T^T E_raw T.  Per deflating instance, on the host: the eigen part is
// orthonormalised (T = [L_r^-T; 0] with G_rr = L_r L_r^T); each candidate e_j
// is orthogonalised against T twice, skipped if its norm is below tau_dep,
// normalised, and accepted while cond(E_trial) <= tau_safe (the first
// violation ends the merge).  The coarse inverse becomes T E_Z^-1 T^T; the
// guard applies to cond(E_Z).
sdf_status safe_merge_select(sdf_problem *p, int B, int k, int r, InstState *st_d,
                             const double *G_d, const double *Eraw_d, double *Einv_d,
                             double tau_safe, double tau_dep, double tau_cond, cudaStream_t s) {
  const size_t kk = (size_t)k * k;
  std::vector<InstState> st(B);
  std::vector<double> Gh((size_t)B * kk), Eh((size_t)B * kk);
  CK(cudaMemcpyAsync(st.data(), st_d, sizeof(InstState) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(Gh.data(), G_d, sizeof(double) * Gh.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(Eh.data(), Eraw_d, sizeof(double) * Eh.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  auto galerkin = [&](const double *E, const std::vector<std::vector<double>> &T) {
    const int m = (int)T.size();
    std::vector<double> out((size_t)m * m, 0.0);
    for (int a = 0; a < m; ++a)
      for (int b2 = 0; b2 < m; ++b2) {
        double v = 0.0;
        for (int i = 0; i < k; ++i) {
          if (T[a][i] == 0.0) continue;
          double w = 0.0;
          for (int j = 0; j < k; ++j) w += E[(size_t)i * k + j] * T[b2][j];
          v += T[a][i] * w;
        }
        out[(size_t)a * m + b2] = v;
      }
    for (int a = 0; a < m; ++a)
      for (int b2 = a + 1; b2 < m; ++b2) {
        const double sy = 0.5 * (out[(size_t)a * m + b2] + out[(size_t)b2 * m + a]);
        out[(size_t)a * m + b2] = out[(size_t)b2 * m + a] = sy;
      }
    return out;
  };
  auto cond_of = [&](std::vector<double> E, int m) {
    std::vector<double> w, V;
    hla::jacobi_eig(m, E, w, V);  // descending
    return w[m - 1] > 0.0 ? w[0] / w[m - 1] : INFINITY;
  };
  std::vector<double> Ei(kk);
  for (int b = 0; b < B; ++b) {
    InstState &S = st[b];
    if (S.outer_done || !S.deflate) continue;
    const double *G = Gh.data() + (size_t)b * kk, *E = Eh.data() + (size_t)b * kk;
    auto Gdot = [&](const std::vector<double> &x, const std::vector<double> &y) {
      double v = 0.0;
      for (int i = 0; i < k; ++i) {
        if (x[i] == 0.0) continue;
        double w = 0.0;
        for (int j = 0; j < k; ++j) w += G[(size_t)i * k + j] * y[j];
        v += x[i] * w;
      }
      return v;
    };
    // eigen part: T = [L_r^-T; 0]
    std::vector<double> Grr((size_t)r * r), Lr, Wr;
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < r; ++j) Grr[(size_t)i * r + j] = G[(size_t)i * k + j];
    bool good = hla::cholesky(r, Grr, Lr);
    std::vector<std::vector<double>> T;
    if (good) {
      hla::inv_lower_transpose(r, Lr, Wr);
      for (int c = 0; c < r; ++c) {
        std::vector<double> t(k, 0.0);
        for (int i = 0; i < r; ++i) t[i] = Wr[(size_t)i * r + c];
        T.push_back(t);
      }
      for (int j = r; j < k; ++j) {
        std::vector<double> c(k, 0.0);
        c[j] = 1.0;
        for (int rep = 0; rep < 2; ++rep) {
          std::vector<double> proj(T.size());
          for (size_t a = 0; a < T.size(); ++a) proj[a] = Gdot(T[a], c);
          for (size_t a = 0; a < T.size(); ++a)
            for (int i = 0; i < k; ++i) c[i] -= proj[a] * T[a][i];
        }
        const double nrm = std::sqrt(std::max(0.0, Gdot(c, c)));
        if (nrm < tau_dep) continue;
        for (int i = 0; i < k; ++i) c[i] /= nrm;
        T.push_back(c);
        const std::vector<double> Et = galerkin(E, T);
        if (!(cond_of(Et, (int)T.size()) <= tau_safe)) {
          T.pop_back();
          break;
        }
      }
    }
    const int m = (int)T.size();
    double cond = INFINITY;
    std::vector<double> EZ, L, Winv;
    if (good) {
      EZ = galerkin(E, T);
      cond = cond_of(EZ, m);
      good = cond <= tau_cond && hla::cholesky(m, EZ, L);
    }
    S.stats.cond_E[S.outer] = cond;
    if (!good) {
      S.deflate = 0;
      S.stats.fallback[S.outer] = 1;
      continue;
    }
    S.stats.fallback[S.outer] = 0;
    // Einv = T E_Z^-1 T^T with E_Z^-1 = W W^T, W = L^-T
    hla::inv_lower_transpose(m, L, Winv);
    std::vector<double> TW((size_t)k * m, 0.0);  // T W (k x m)
    for (int i = 0; i < k; ++i)
      for (int c = 0; c < m; ++c) {
        double v = 0.0;
        for (int a = 0; a < m; ++a) v += T[a][i] * Winv[(size_t)a * m + c];
        TW[(size_t)i * m + c] = v;
      }
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        double v = 0.0;
        for (int c = 0; c < m; ++c) v += TW[(size_t)i * m + c] * TW[(size_t)j * m + c];
        Ei[(size_t)i * k + j] = v;
      }
    CK(cudaMemcpyAsync(Einv_d + (size_t)b * kk, Ei.data(), sizeof(double) * kk,
                       cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  CK(cudaMemcpyAsync(st_d, st.data(), sizeof(InstState) * B, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return SDF_OK;
}

// Ritz re-selection (Sec. 2.2.3) after k_coarse: for each deflating
// instance, the eigenpairs (mu, C) of E = Lg^-1 E_raw Lg^-T (the Galerkin
// matrix of the orthonormalised pool Phi_I Lg^-T) on the host; the r
// smallest are kept, the guard is applied to mu_r / mu_1, and the coarse
// inverse becomes Einv = Lg^-T C_r diag(1/mu) C_r^T Lg^-1, i.e. the A-DEF2
// projector of Z = Phi_I Lg^-T C_r.  coarse holds (Lg, Lg^-1, T, E, Le^-1)
// per instance, row-major.
sdf_status ritz_select(sdf_problem *p, int B, int k, int r, InstState *st_d, const double *coarse_d,
                       double *Einv_d, double tau_cond, cudaStream_t s) {
  const size_t kk = (size_t)k * k;
  std::vector<InstState> st(B);
  std::vector<double> cs((size_t)B * 5 * kk);
  CK(cudaMemcpyAsync(st.data(), st_d, sizeof(InstState) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(cs.data(), coarse_d, sizeof(double) * cs.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<double> Ei(kk);
  for (int b = 0; b < B; ++b) {
    InstState &S = st[b];
    if (S.outer_done || !S.deflate) continue;
    const double *Lgi = cs.data() + (size_t)b * 5 * kk + kk;
    std::vector<double> E(cs.begin() + (size_t)b * 5 * kk + 3 * kk,
                          cs.begin() + (size_t)b * 5 * kk + 4 * kk), w, Vd;
    hla::jacobi_eig(k, E, w, Vd);  // descending
    const double mu1 = w[k - 1], mur = w[k - r];
    const double cond = mu1 > 0.0 ? mur / mu1 : INFINITY;
    S.stats.cond_E[S.outer] = cond;
    if (!(cond <= tau_cond)) {
      S.deflate = 0;
      S.stats.fallback[S.outer] = 1;
      continue;
    }
    // Y = C_r^T Lg^-1 (r x k); Einv = Y^T diag(1 / mu) Y
    std::vector<double> Y((size_t)r * k, 0.0);
    for (int a = 0; a < r; ++a) {
      const int col = k - 1 - a;  // a-th smallest
      for (int j = 0; j < k; ++j) {
        double v = 0.0;
        for (int q = 0; q < k; ++q) v += Vd[(size_t)q * k + col] * Lgi[(size_t)q * k + j];
        Y[(size_t)a * k + j] = v;
      }
    }
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        double v = 0.0;
        for (int a = 0; a < r; ++a) v += Y[(size_t)a * k + i] * Y[(size_t)a * k + j] / w[k - 1 - a];
        Ei[(size_t)i * k + j] = v;
      }
    CK(cudaMemcpyAsync(Einv_d + (size_t)b * kk, Ei.data(), sizeof(double) * kk,
                       cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  CK(cudaMemcpyAsync(st_d, st.data(), sizeof(InstState) * B, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return SDF_OK;
}

// A chunk of CG launches (the iterations between two host polls, and on the
// mixed path the residual replacement and correction pass after them),
// captured once per solve call into a CUDA graph on a private stream and
// replayed on the caller's stream: one slot per starting parity of the
// ping-pong residual buffers.  Capturing launches nothing, so the host-side
// effects of the captured body (parity flips, launch counts) are undone and
// then applied per replay.
struct ChunkGraphs {
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  int flip[2] = {0, 0};
  long long launches[2] = {0, 0};
  ~ChunkGraphs() {
    for (cudaGraphExec_t &e : exec)
      if (e) cudaGraphExecDestroy(e);
  }
};

// body(stream) enqueues one chunk on `stream`, advancing *par and the
// problem's launch count.  use_graph = false launches it directly on s.
template <class Body>
sdf_status run_chunk(sdf_problem *p, ChunkGraphs &gr, bool use_graph, cudaStream_t s, int *par,
                     Body body) {
  if (!use_graph) return body(s);
  const int slot = *par & 1;
  if (!gr.exec[slot]) {
    if (!p->cap_stream) CK(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    const int par0 = *par;
    const long long l0 = p->prof.launches;
    CK(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    const sdf_status e = body(p->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &g);
    if (e != SDF_OK) {
      if (g) cudaGraphDestroy(g);
      return e;
    }
    CK(ce);
    const cudaError_t ie = cudaGraphInstantiate(&gr.exec[slot], g, 0);
    cudaGraphDestroy(g);
    CK(ie);
    gr.flip[slot] = (*par ^ par0) & 1;
    gr.launches[slot] = p->prof.launches - l0;
    *par = par0;
    p->prof.launches = l0;
  }
  CK(cudaGraphLaunch(gr.exec[slot], s));
  *par ^= gr.flip[slot];
  p->prof.launches += gr.launches[slot];
  return SDF_OK;
}

template <int DIM, int KMAX, class PhiT, class V>
sdf_status solve_impl(sdf_problem *p, const double *inst, int B, const double *psi,
                      const sdf_opts &o, char *ws, cudaStream_t s, double *y, double *lam,
                      uint8_t *active, sdf_stats *stats) {
  constexpr int mixed = sizeof(V) == sizeof(float) ? 1 : 0;
  const Layout L = make_layout(p, B, o.max_blocks, mixed);
  const OpParams &P = p->P;
  const long long N = P.N;
  double *x = (double *)(ws + L.x), *b64 = (double *)(ws + L.b64);
  V *pp = (V *)(ws + L.p), *q = (V *)(ws + L.q);
  V *rbuf[2] = {(V *)(ws + L.r), (V *)(ws + L.r2)};
  V *dinv = P.convection ? (V *)(ws + L.dinv)
                         : (mixed ? (V *)p->dinv_shared32 : (V *)p->dinv_shared);
  uint8_t *mask = (uint8_t *)(ws + L.mask);
  double *W = (double *)(ws + L.W), *Einv = (double *)(ws + L.Einv), *Eraw = (double *)(ws + L.Eraw),
         *G = (double *)(ws + L.G), *coarse = (double *)(ws + L.coarse),
         *part = (double *)(ws + L.part), *gpart = (double *)(ws + L.gpart);
  InstState *st = (InstState *)(ws + L.state);
  int *cnt = (int *)(ws + L.cnt);
  Ctrl *ctrl = (Ctrl *)(ws + L.ctrl);
  const bool defl = o.deflate && p->phi != nullptr && p->k > 0;
  const int k = defl ? p->k : 0;
  const PhiT *Phi = phi_as<PhiT>(p);
  const long long ld = p->ld;
  // shared-Phi batch kernels: v = S z - r written by the update, projected for
  // the whole batch by one GEMM, expanded per node for groups of instances
  constexpr bool f64 = std::is_same<PhiT, double>::value && std::is_same<V, double>::value;
  const bool fb = f64 && defl && L.fb;
  V *vv = (V *)(ws + L.v);
  double *cvec64 = (double *)(ws + L.cvec), *ppart64 = (double *)(ws + L.ppart);
  const dim3 gPb(L.bpad / std::max(L.nb, 1), L.gxp);
  const int ngrp = (B + kExpandGroup - 1) / kExpandGroup;
  const dim3 gEb(ngrp, (int)std::max<long long>(
                           1, std::min<long long>((N + NT - 1) / NT, (p->nsm * 4LL + ngrp - 1) / ngrp)));

  CK(cudaMemsetAsync(mask, 0, (size_t)N * B, s));
  CK(cudaMemsetAsync(st, 0, sizeof(InstState) * B, s));
  CK(cudaMemsetAsync(cnt, 0, sizeof(int) * B * NCNT, s));
  CK(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s));
  if (fb) CK(cudaMemsetAsync(cvec64, 0, sizeof(double) * B * KMAX, s));

  cudaStream_t ls = s;  // stream of the CG launches (a capture stream while a chunk is captured)
  ChunkGraphs graphs;
  // cvec64 <- csign E^-1 Phi_I^T src for every running instance (batch kernels)
  auto project64 = [&](const V *src) -> sdf_status {
    if constexpr (f64) {
      switch (L.nb) {
        case 16: k_proj_gemm64<KMAX, 16><<<gPb, NT, 0, ls>>>(Phi, ld, k, N, B, st, src, ppart64, L.bpad); break;
        case 32: k_proj_gemm64<KMAX, 32><<<gPb, NT, 0, ls>>>(Phi, ld, k, N, B, st, src, ppart64, L.bpad); break;
        default: k_proj_gemm64<KMAX, 64><<<gPb, NT, 0, ls>>>(Phi, ld, k, N, B, st, src, ppart64, L.bpad); break;
      }
      k_proj_reduce<KMAX, double><<<B, NT, 0, ls>>>(ppart64, L.gxp, L.bpad, k, st, Einv, cvec64);
      p->prof.launches += 2;
    }
    return SDF_OK;
  };

  const dim3 gT(B, L.gx), gA(B, L.gxa);
  long long launches = 0;
  const long long max_launches = o.max_launches > 0 ? o.max_launches : 4LL * o.max_cg + 64;
  // CG iterations between FP64 residual replacements (mixed) or host polls
  const int chunk = std::max(1, mixed ? (o.replace_every > 0 ? o.replace_every : 100) : o.check_every);
  const double rtol2 = o.rtol * o.rtol;
  const double floor_cu = std::max(o.floor_c, 0.0) * std::ldexp(1.0, -53);
  int live = B;
  int par = 0;
  // one CG-kernel triple: A (expand into `dir`), B (spmv of dir), C (update)
  auto triple = [&](V *dir, bool timed) -> sdf_status {
    if (timed) CK(cudaEventRecord(p->ev[0], s));
    bool expanded = false;
    if constexpr (f64) {
      if (fb) {
        k_expand64_b<KMAX, kExpandGroup><<<gEb, NT, 0, ls>>>(Phi, ld, k, N, B, st, cvec64, mask,
                                                            rbuf[par], dinv, P.convection, dir);
        expanded = true;
      }
    }
    if (!expanded)
      k_expand<KMAX, PhiT, V><<<gA, NT, 0, ls>>>(Phi, ld, k, N, st, Einv, mask, rbuf[par], dinv,
                                                P.convection, dir, L.gxa);
    if (timed) CK(cudaEventRecord(p->ev[1], s));
    k_spmv<DIM, V><<<gT, NT, 0, ls>>>(P, inst, st, mask, dir, q, part, cnt, ctrl, L.gx);
    if (timed) CK(cudaEventRecord(p->ev[2], s));
    k_update<DIM, KMAX, PhiT, V><<<gT, NT, 0, ls>>>(P, inst, Phi, ld, k, st, mask, rbuf[par],
                                                   rbuf[par ^ 1], q, dir, x, dinv, part, cnt,
                                                   ctrl, L.gx, rtol2, o.max_cg, mixed,
                                                   fb ? vv : nullptr);
    if (timed) CK(cudaEventRecord(p->ev[3], s));
    if (fb) {
      sdf_status e = project64(vv);
      if (e != SDF_OK) return e;
    }
    if (timed && fb) CK(cudaEventRecord(p->ev[4], s));
    par ^= 1;
    p->prof.launches += 3;
    return SDF_OK;
  };
  for (int outer = 0; outer < o.max_outer && live > 0; ++outer) {
    CK(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s));
    par = 0;
    k_outer_setup<DIM, V><<<gT, NT, 0, s>>>(P, inst, psi, mask, rbuf[0], b64, x, dinv, st, part,
                                            cnt, ctrl, L.gx, p->x0, y);
    CKL("k_outer_setup");
    p->prof.launches += 1;
    if (p->x0) {
      k_start_resid<DIM, V><<<gT, NT, 0, s>>>(P, inst, st, mask, b64, x, rbuf[0], L.gx);
      CKL("k_start_resid");
      p->prof.launches += 1;
    }
    if (defl) {
      // The first outer iteration of every instance has A = {} (cold start);
      // without per-instance convection S_II and Phi_I are then the same for
      // the whole batch, and so are E_raw and G: set up once, copied.
      const int nset = (outer == 0 && !P.convection) ? 1 : B;
      for (int b = 0; b < nset; ++b) {
        k_modes_W<DIM, PhiT><<<dim3(k, L.gx), NT, 0, s>>>(P, inst, b, st, mask, Phi, ld, W, L.gx);
        k_gram<KMAX, PhiT><<<L.gxg, NT, 0, s>>>(Phi, ld, W, mask, st, b, N, k, 0, gpart);
        k_gram_reduce<<<(k * k + NT - 1) / NT, NT, 0, s>>>(gpart, L.gxg, k, st, b, Eraw + (size_t)b * k * k);
        k_gram<KMAX, PhiT><<<L.gxg, NT, 0, s>>>(Phi, ld, W, mask, st, b, N, k, 1, gpart);
        k_gram_reduce<<<(k * k + NT - 1) / NT, NT, 0, s>>>(gpart, L.gxg, k, st, b, G + (size_t)b * k * k);
      }
      if (nset < B)
        k_coarse_copy<<<B - 1, NT, 0, s>>>(k, Eraw, G);
      CKL("coarse setup");
      {
        const bool merge = o.safe_r > 0 && o.safe_r < k;
        const bool ritz = !merge && o.ritz_r > 0 && o.ritz_r < k;
        k_coarse<<<B, NT, 0, s>>>(k, st, G, Eraw, Einv, coarse,
                                  (ritz || merge) ? INFINITY : o.tau_cond, merge ? 1 : 0);
        CKL("k_coarse");
        if (merge) {
          sdf_status e = safe_merge_select(p, B, k, o.safe_r, st, G, Eraw, Einv, o.tau_safe,
                                           o.tau_dep, o.tau_cond, s);
          if (e != SDF_OK) return e;
        } else if (ritz) {
          sdf_status e = ritz_select(p, B, k, o.ritz_r, st, coarse, Einv, o.tau_cond, s);
          if (e != SDF_OK) return e;
        }
      }
      if (fb) {
        sdf_status e = project64(rbuf[0]);  // coarse-corrected start: c = -E^-1 Phi_I^T b
        if (e != SDF_OK) return e;
      } else {
        k_project<KMAX, PhiT, V><<<gA, NT, 0, s>>>(Phi, ld, k, N, mask, rbuf[0], st, nullptr,
                                                   part, cnt, L.gxa);
        p->prof.launches += 1;
      }
      CKL("k_project");
      p->prof.launches += 5LL * nset + (nset < B ? 1 : 0) + 1;
    }
    // coarse-corrected start (phase 1), then CG iterations in chunks; r
    // ping-pongs between its two buffers (uniform across the batch: finished
    // instances skip every launch).
    {
      sdf_status e = triple(pp, false);
      if (e != SDF_OK) return e;
    }
    for (int it = 0;; ++it) {
      const bool timed = o.profile && p->ev_ready;
      sdf_status e = run_chunk(p, graphs, o.graph != 0 && !timed, s, &par,
                               [&](cudaStream_t cs) -> sdf_status {
                                 ls = cs;
                                 for (int rep = 0; rep < chunk; ++rep) {
                                   const sdf_status e2 = triple(pp, timed && rep == 0);
                                   if (e2 != SDF_OK) {
                                     ls = s;
                                     return e2;
                                   }
                                 }
                                 ls = s;
                                 return SDF_OK;
                               });
      if (e != SDF_OK) return e;
      CKL("cg iteration");
      launches += chunk;
      CK(cudaMemcpyAsync(p->pinned, &ctrl->running, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (timed) {
        float t0 = 0, t1 = 0, t2 = 0, t3 = 0;
        cudaEventElapsedTime(&t0, p->ev[0], p->ev[1]);
        cudaEventElapsedTime(&t1, p->ev[1], p->ev[2]);
        cudaEventElapsedTime(&t2, p->ev[2], p->ev[3]);
        if (mixed) cudaEventElapsedTime(&t3, p->ev[4], p->ev[5]);
        float t4 = 0;
        if (fb) cudaEventElapsedTime(&t4, p->ev[3], p->ev[4]);
        // only intervals that still had work count (a poll interval whose first
        // iteration found every instance finished would time empty launches)
        if (p->pinned[0] > 0 || chunk > 1) {
          p->prof.ms[0] += t0;
          p->prof.ms[1] += t1;
          p->prof.ms[2] += t2;
          p->prof.samples[0] += 1;
          p->prof.samples[1] += 1;
          p->prof.samples[2] += 1;
          if (mixed) {
            p->prof.ms[7] += t3;
            p->prof.samples[7] += 1;
          }
          if (fb) {
            p->prof.ms[8] += t4;
            p->prof.samples[8] += 1;
          }
        }
      }
      if (p->pinned[0] <= 0) break;
      if (launches > max_launches)
        return fail(p, SDF_ERR_TIMEOUT, "solve exceeded its iteration launch budget");
    }
    k_exit_resid<DIM><<<gT, NT, 0, s>>>(P, inst, st, mask, b64, x, nullptr, part, cnt, L.gx,
                                        floor_cu);
    CKL("k_exit_resid");
    k_active<<<gA, NT, 0, s>>>(N, psi, mask, x, nullptr, y, st, part, cnt, ctrl, L.gxa, o.tau,
                               o.max_outer);
    CKL("k_active");
    p->prof.launches += 2;  // k_exit_resid, k_active
    CK(cudaMemcpyAsync(p->pinned + 1, &ctrl->live, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    live = p->pinned[1];
  }
  if (active) CK(cudaMemcpyAsync(active, mask, (size_t)N * B, cudaMemcpyDeviceToDevice, s));
  if (lam) {
    k_lambda<DIM><<<gT, NT, 0, s>>>(P, inst, y, lam, L.gx);
    CKL("k_lambda");
    p->prof.launches += 1;
  }
  std::vector<InstState> hs(B);
  CK(cudaMemcpyAsync(hs.data(), st, sizeof(InstState) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int worst = SDF_OK;
  for (int b = 0; b < B; ++b) {
    if (stats) stats[b] = hs[b].stats;
    if (hs[b].stats.status != SDF_OK && worst == SDF_OK) worst = hs[b].stats.status;
  }
  if (worst != SDF_OK) p->err = "at least one instance did not converge (see stats)";
  return (sdf_status)worst;
}

// Mixed-precision solve (SDF_PREC_MIXED): FP32 vectors, stencil and
// shared-Phi kernels; FP64 iterate, right-hand side, reductions, coarse
// operator and periodic residual replacement (k_resid) with coarse correction.
template <int DIM, int KMAX, class PhiT>
sdf_status solve_mixed(sdf_problem *p, const double *inst, int B, const double *psi,
                       const sdf_opts &o, char *ws, cudaStream_t s, double *y, double *lam,
                       uint8_t *active, sdf_stats *stats) {
  const Layout L = make_layout(p, B, o.max_blocks, 1, o.column_depth, o.column_pairs);
  const OpParams &P = p->P;
  const long long N = P.N;
  double *x = (double *)(ws + L.x), *b64 = (double *)(ws + L.b64);
  float *pp = (float *)(ws + L.p), *q = (float *)(ws + L.q), *wv = (float *)(ws + L.w);
  float *vv = (float *)(ws + L.v), *cvec = (float *)(ws + L.cvec), *xlo = (float *)(ws + L.xlo);
  double *ppart = (double *)(ws + L.ppart);
  float *rbuf[2] = {(float *)(ws + L.r), (float *)(ws + L.r2)};
  float *dinv = P.convection ? (float *)(ws + L.dinv) : p->dinv_shared32;
  uint8_t *mask = (uint8_t *)(ws + L.mask);
  double *W = (double *)(ws + L.W), *Einv = (double *)(ws + L.Einv), *Eraw = (double *)(ws + L.Eraw),
         *G = (double *)(ws + L.G), *coarse = (double *)(ws + L.coarse),
         *part = (double *)(ws + L.part), *gpart = (double *)(ws + L.gpart);
  InstState *st = (InstState *)(ws + L.state);
  int *cnt = (int *)(ws + L.cnt);
  Ctrl *ctrl = (Ctrl *)(ws + L.ctrl);
  const bool defl = o.deflate && p->phi != nullptr && p->k > 0;
  const int k = defl ? p->k : 0;
  const PhiT *Phi = phi_as<PhiT>(p);
  const long long ld = p->ld;

  CK(cudaMemsetAsync(mask, 0, (size_t)N * B, s));
  CK(cudaMemsetAsync(st, 0, sizeof(InstState) * B, s));
  CK(cudaMemsetAsync(cnt, 0, sizeof(int) * B * NCNT, s));
  CK(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s));
  CK(cudaMemsetAsync(cvec, 0, sizeof(float) * B * KMAX, s));

  const size_t esm = sizeof(float) * (size_t)B * KMAX + 3 * sizeof(float) * B;
  if (esm > 48 * 1024)
    CK(cudaFuncSetAttribute(k_expand_b<KMAX, PhiT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)esm));
  const dim3 gT(B, L.gx);
  const int gxe = (int)std::max<long long>(1, std::min<long long>((N + NT - 1) / NT, p->nsm * 4LL));
  const dim3 gP((B + L.nb - 1) / L.nb, L.gxp);
  long long launches = 0;
  const long long max_launches = o.max_launches > 0 ? o.max_launches : 4LL * o.max_cg + 64;
  const int chunk = std::max(1, o.replace_every > 0 ? o.replace_every : 100);
  const double rtol2 = o.rtol * o.rtol;
  const double floor_cu = std::max(o.floor_c, 0.0) * std::ldexp(1.0, -53);
  int live = B;
  int par = 0;
  __nv_bfloat16 *phin = (__nv_bfloat16 *)(ws + L.phin);
  const size_t xsm = expand_tc_smem(L.nbp, L.kp);
  const int gxt = (int)std::max<long long>(1, std::min<long long>((N + 127) / 128, p->nsm * 6LL));
  if constexpr (std::is_same<PhiT, __nv_bfloat16>::value) {
    if (L.tce && defl) {
      k_phi_node_major<<<p->nsm * 8, NT, 0, s>>>(Phi, ld, k, N, L.kp, phin);
      CKL("k_phi_node_major");
      cudaError_t e = cudaSuccess;
      switch (L.nbp) {
        case 16: e = cudaFuncSetAttribute(k_expand_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm); break;
        case 32: e = cudaFuncSetAttribute(k_expand_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm); break;
        case 64: e = cudaFuncSetAttribute(k_expand_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm); break;
        case 128: e = cudaFuncSetAttribute(k_expand_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm); break;
        default: e = cudaFuncSetAttribute(k_expand_tc<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm); break;
      }
      CK(e);
    }
    if (L.tcp && defl) {  // the larger batch tiles need more than 48 KB of shared memory
      const int sm = tc::GM * tc::GK * 2 + 3 * L.nbp * tc::GK * 2;
      cudaError_t e = cudaSuccess;
      switch (L.nbp) {
        case 16: e = cudaFuncSetAttribute(k_proj_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm); break;
        case 32: e = cudaFuncSetAttribute(k_proj_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm); break;
        case 64: e = cudaFuncSetAttribute(k_proj_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm); break;
        case 128: e = cudaFuncSetAttribute(k_proj_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm); break;
        default: e = cudaFuncSetAttribute(k_proj_tc<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm); break;
      }
      CK(e);
    }
  }
  cudaStream_t ls = s;  // stream of the CG launches (a capture stream while a chunk is captured)
  ChunkGraphs graphs;
  auto project = [&](const float *src) -> sdf_status {  // cvec <- csign E^-1 Phi_I^T src
    if (!defl) return SDF_OK;
    if constexpr (std::is_same<PhiT, __nv_bfloat16>::value) {
      if (L.tcp) {
        const size_t sm = (size_t)tc::GM * tc::GK * 2 + 3 * (size_t)L.nbp * tc::GK * 2;
        switch (L.nbp) {
          case 16: k_proj_tc<16><<<L.gxp, tc::GTH, sm, ls>>>(Phi, ld, k, N, B, st, src, ppart, L.bpad, KMAX); break;
          case 32: k_proj_tc<32><<<L.gxp, tc::GTH, sm, ls>>>(Phi, ld, k, N, B, st, src, ppart, L.bpad, KMAX); break;
          case 64: k_proj_tc<64><<<L.gxp, tc::GTH, sm, ls>>>(Phi, ld, k, N, B, st, src, ppart, L.bpad, KMAX); break;
          case 128: k_proj_tc<128><<<L.gxp, tc::GTH, sm, ls>>>(Phi, ld, k, N, B, st, src, ppart, L.bpad, KMAX); break;
          default: k_proj_tc<256><<<L.gxp, tc::GTH, sm, ls>>>(Phi, ld, k, N, B, st, src, ppart, L.bpad, KMAX); break;
        }
        k_proj_reduce<KMAX><<<B, NT, 0, ls>>>(ppart, L.gxp, L.bpad, k, st, Einv, cvec);
        p->prof.launches += 2;
        return SDF_OK;
      }
    }
    if (L.nb == 1)
      k_proj_gemm<KMAX, 1, PhiT><<<gP, NT, 0, ls>>>(Phi, ld, k, N, B, st, src, ppart, L.bpad);
    else if (L.nb == 16)
      k_proj_gemm<KMAX, 16, PhiT><<<gP, NT, 0, ls>>>(Phi, ld, k, N, B, st, src, ppart, L.bpad);
    else if (L.nb == 32)
      k_proj_gemm<KMAX, 32, PhiT><<<gP, NT, 0, ls>>>(Phi, ld, k, N, B, st, src, ppart, L.bpad);
    else
      k_proj_gemm<KMAX, 64, PhiT><<<gP, NT, 0, ls>>>(Phi, ld, k, N, B, st, src, ppart, L.bpad);
    k_proj_reduce<KMAX><<<B, NT, 0, ls>>>(ppart, L.gxp, L.bpad, k, st, Einv, cvec);
    p->prof.launches += 2;
    return SDF_OK;
  };
  auto triple = [&](float *dir, bool timed) -> sdf_status {
    if (timed) CK(cudaEventRecord(p->ev[0], s));
    bool expanded = false;
    if constexpr (std::is_same<PhiT, __nv_bfloat16>::value) {
      if (L.tce && defl) {
#define SDF_EXPAND_TC(NB_)                                                                        \
  k_expand_tc<NB_><<<gxt, tc::GTH, xsm, ls>>>(phin, L.kp, N, B, st, cvec, KMAX, mask, rbuf[par], \
                                             dinv, P.convection, dir)
        switch (L.nbp) {
          case 16: SDF_EXPAND_TC(16); break;
          case 32: SDF_EXPAND_TC(32); break;
          case 64: SDF_EXPAND_TC(64); break;
          case 128: SDF_EXPAND_TC(128); break;
          default: SDF_EXPAND_TC(256); break;
        }
#undef SDF_EXPAND_TC
        expanded = true;
      }
    }
    if (!expanded)
      k_expand_b<KMAX, PhiT><<<gxe, NT, esm, ls>>>(Phi, ld, k, N, B, st, cvec, mask, rbuf[par],
                                                  dinv, P.convection, dir);
    if (timed) CK(cudaEventRecord(p->ev[1], s));
    if constexpr (DIM == 3) {
      // the mixed path has no convection (rejected at entry): VARK only
      if (L.pairs) {  // instance pairs on the packed FP32 pipe
        // column items fastest: the blocks resident at one time hold every
        // item of a few pairs, so neighbouring tiles read each other's halo
        // sectors from L2 while both march the same planes
        const dim3 gC2(L.gxc, (B + 1) / 2);
        auto spmv = P.fx ? k_spmv3p<true> : k_spmv3p<false>;
        auto upd = P.fx ? k_update_v3p<true> : k_update_v3p<false>;
        spmv<<<gC2, NT, 0, ls>>>(P, st, mask, dir, q, part, cnt, ctrl, L.gxc, L.zc, B);
        if (timed) CK(cudaEventRecord(p->ev[2], s));
        upd<<<gC2, NT, 0, ls>>>(P, st, mask, rbuf[par], rbuf[par ^ 1], q, dir, x, xlo, dinv, vv,
                               part, cnt, ctrl, L.gxc, L.zc, rtol2, o.max_cg, B);
      } else {
        const dim3 gC(B, L.gxc);
        auto spmv = P.fx ? k_spmv3c<true> : k_spmv3c<false>;
        auto upd = P.fx ? k_update_v3c<true> : k_update_v3c<false>;
        spmv<<<gC, NT, 0, ls>>>(P, inst, st, mask, dir, q, part, cnt, ctrl, L.gxc, L.zc);
        if (timed) CK(cudaEventRecord(p->ev[2], s));
        upd<<<gC, NT, 0, ls>>>(P, inst, st, mask, rbuf[par], rbuf[par ^ 1], q, dir, x, xlo, dinv,
                              vv, part, cnt, ctrl, L.gxc, L.zc, rtol2, o.max_cg);
      }
    } else {
      k_spmv<DIM, float><<<gT, NT, 0, ls>>>(P, inst, st, mask, dir, q, part, cnt, ctrl, L.gx);
      if (timed) CK(cudaEventRecord(p->ev[2], s));
      k_update_v<DIM><<<gT, NT, 0, ls>>>(P, inst, st, mask, rbuf[par], rbuf[par ^ 1], q, dir, x,
                                        xlo, dinv, vv, part, cnt, ctrl, L.gx, rtol2, o.max_cg);
    }
    if (timed) CK(cudaEventRecord(p->ev[3], s));
    sdf_status e = project(vv);
    if (e != SDF_OK) return e;
    if (timed) CK(cudaEventRecord(p->ev[4], s));
    par ^= 1;
    p->prof.launches += 3;
    return SDF_OK;
  };
  for (int outer = 0; outer < o.max_outer && live > 0; ++outer) {
    CK(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s));
    CK(cudaMemsetAsync(xlo, 0, sizeof(float) * (size_t)N * B, s));
    par = 0;
    k_outer_setup<DIM, float><<<gT, NT, 0, s>>>(P, inst, psi, mask, rbuf[0], b64, x, dinv, st,
                                                part, cnt, ctrl, L.gx, p->x0, y);
    CKL("k_outer_setup");
    p->prof.launches += 1;
    if (p->x0) {
      k_start_resid<DIM, float><<<gT, NT, 0, s>>>(P, inst, st, mask, b64, x, rbuf[0], L.gx);
      CKL("k_start_resid");
      p->prof.launches += 1;
    }
    if (defl) {
      // The first outer iteration of every instance has A = {} (cold start);
      // without per-instance convection S_II and Phi_I are then the same for
      // the whole batch, and so are E_raw and G: set up once, copied.
      const int nset = (outer == 0 && !P.convection) ? 1 : B;
      for (int b = 0; b < nset; ++b) {
        k_modes_W<DIM, PhiT><<<dim3(k, L.gx), NT, 0, s>>>(P, inst, b, st, mask, Phi, ld, W, L.gx);
        k_gram<KMAX, PhiT><<<L.gxg, NT, 0, s>>>(Phi, ld, W, mask, st, b, N, k, 0, gpart);
        k_gram_reduce<<<(k * k + NT - 1) / NT, NT, 0, s>>>(gpart, L.gxg, k, st, b, Eraw + (size_t)b * k * k);
        k_gram<KMAX, PhiT><<<L.gxg, NT, 0, s>>>(Phi, ld, W, mask, st, b, N, k, 1, gpart);
        k_gram_reduce<<<(k * k + NT - 1) / NT, NT, 0, s>>>(gpart, L.gxg, k, st, b, G + (size_t)b * k * k);
      }
      if (nset < B)
        k_coarse_copy<<<B - 1, NT, 0, s>>>(k, Eraw, G);
      CKL("coarse setup");
      {
        const bool merge = o.safe_r > 0 && o.safe_r < k;
        const bool ritz = !merge && o.ritz_r > 0 && o.ritz_r < k;
        k_coarse<<<B, NT, 0, s>>>(k, st, G, Eraw, Einv, coarse,
                                  (ritz || merge) ? INFINITY : o.tau_cond, merge ? 1 : 0);
        CKL("k_coarse");
        if (merge) {
          sdf_status e = safe_merge_select(p, B, k, o.safe_r, st, G, Eraw, Einv, o.tau_safe,
                                           o.tau_dep, o.tau_cond, s);
          if (e != SDF_OK) return e;
        } else if (ritz) {
          sdf_status e = ritz_select(p, B, k, o.ritz_r, st, coarse, Einv, o.tau_cond, s);
          if (e != SDF_OK) return e;
        }
      }
      p->prof.launches += 5LL * nset + (nset < B ? 1 : 0) + 1;
      sdf_status e = project(rbuf[0]);  // coarse-corrected start: c = -E^-1 Phi_I^T b
      if (e != SDF_OK) return e;
    }
    {
      sdf_status e = triple(pp, false);  // phase 1
      if (e != SDF_OK) return e;
    }
    for (;;) {
      const bool timed = o.profile && p->ev_ready;
      // one chunk: `chunk` CG iterations, the FP64 residual replacement and
      // the correction pass
      sdf_status ec = run_chunk(p, graphs, o.graph != 0 && !timed, s, &par,
                                [&](cudaStream_t cs) -> sdf_status {
        ls = cs;
        for (int rep = 0; rep < chunk; ++rep) {
          sdf_status e = triple(pp, timed && rep == 0);
          if (e != SDF_OK) {
            ls = s;
            return e;
          }
        }
        if (timed) CK(cudaEventRecord(p->ev[5], s));
        if constexpr (DIM == 3)
          k_resid<DIM><<<dim3(B, L.gxc), NT, 0, ls>>>(P, inst, st, mask, b64, x, xlo, rbuf[par],
                                                      part, cnt, ctrl, L.gxc, rtol2, floor_cu, L.zc);
        else
          k_resid<DIM><<<gT, NT, 0, ls>>>(P, inst, st, mask, b64, x, xlo, rbuf[par], part, cnt,
                                          ctrl, L.gx, rtol2, floor_cu, L.zc);
        if (timed) CK(cudaEventRecord(p->ev[6], s));
        p->prof.launches += 1;
        sdf_status e = project(rbuf[par]);  // correction pass: c = -E^-1 Phi_I^T r
        if (e == SDF_OK) e = triple(wv, false);
        ls = s;
        return e;
      });
      if (ec != SDF_OK) return ec;
      CKL("cg iteration");
      launches += chunk;
      CK(cudaMemcpyAsync(p->pinned, &ctrl->running, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (timed) {
        float t[6] = {0, 0, 0, 0, 0, 0};
        for (int i = 0; i < 4; ++i) cudaEventElapsedTime(&t[i], p->ev[i], p->ev[i + 1]);
        cudaEventElapsedTime(&t[4], p->ev[5], p->ev[6]);
        const int ids[5] = {0, 1, 2, 8, 7};
        for (int i = 0; i < 5; ++i) {
          p->prof.ms[ids[i]] += t[i];
          p->prof.samples[ids[i]] += 1;
        }
      }
      if (p->pinned[0] <= 0) break;
      if (launches > max_launches)
        return fail(p, SDF_ERR_TIMEOUT, "solve exceeded its iteration launch budget");
    }
    k_exit_resid<DIM><<<gT, NT, 0, s>>>(P, inst, st, mask, b64, x, xlo, part, cnt, L.gx, floor_cu);
    CKL("k_exit_resid");
    k_active<<<dim3(B, L.gxa), NT, 0, s>>>(N, psi, mask, x, xlo, y, st, part, cnt, ctrl, L.gxa,
                                           o.tau, o.max_outer);
    CKL("k_active");
    p->prof.launches += 2;  // k_exit_resid, k_active
    CK(cudaMemcpyAsync(p->pinned + 1, &ctrl->live, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    live = p->pinned[1];
  }
  if (active) CK(cudaMemcpyAsync(active, mask, (size_t)N * B, cudaMemcpyDeviceToDevice, s));
  if (lam) {
    k_lambda<DIM><<<gT, NT, 0, s>>>(P, inst, y, lam, L.gx);
    CKL("k_lambda");
    p->prof.launches += 1;
  }
  std::vector<InstState> hs(B);
  CK(cudaMemcpyAsync(hs.data(), st, sizeof(InstState) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int worst = SDF_OK;
  for (int b = 0; b < B; ++b) {
    if (stats) stats[b] = hs[b].stats;
    if (hs[b].stats.status != SDF_OK && worst == SDF_OK) worst = hs[b].stats.status;
  }
  if (worst != SDF_OK) p->err = "at least one instance did not converge (see stats)";
  return (sdf_status)worst;
}

template <int DIM, int KMAX>
sdf_status dispatch_phi(sdf_problem *p, const double *inst, int B, const double *psi,
                        const sdf_opts &o, char *ws, cudaStream_t s, double *y, double *lam,
                        uint8_t *active, sdf_stats *stats) {
  if (o.precision == SDF_PREC_F64) {
    if (p->phi && p->phi_dtype != SDF_F64 && o.deflate)
      return fail(p, SDF_ERR_UNSUPPORTED, "the FP64 path takes FP64 reference modes");
    return solve_impl<DIM, KMAX, double, double>(p, inst, B, psi, o, ws, s, y, lam, active, stats);
  }
  if constexpr (DIM == 1) {  // refused at entry: a problem given by its operator is FP64 only
    return fail(p, SDF_ERR_UNSUPPORTED, "no mixed path for a problem given by its operator");
  } else {
  switch (p->phi_dtype) {
    case SDF_F32: return solve_mixed<DIM, KMAX, float>(p, inst, B, psi, o, ws, s, y, lam, active, stats);
    case SDF_BF16: return solve_mixed<DIM, KMAX, __nv_bfloat16>(p, inst, B, psi, o, ws, s, y, lam, active, stats);
    default:
      if (p->phi && o.deflate)
        return fail(p, SDF_ERR_UNSUPPORTED, "the mixed path takes FP32 or BF16 reference modes");
      return solve_mixed<DIM, KMAX, float>(p, inst, B, psi, o, ws, s, y, lam, active, stats);
  }
  }
}

template <int DIM>
sdf_status dispatch_k(sdf_problem *p, const double *inst, int B, const double *psi,
                      const sdf_opts &o, char *ws, cudaStream_t s, double *y, double *lam,
                      uint8_t *active, sdf_stats *stats) {
  switch (kmax_for(std::max(p->k, 1))) {
    case 16: return dispatch_phi<DIM, 16>(p, inst, B, psi, o, ws, s, y, lam, active, stats);
    case 32: return dispatch_phi<DIM, 32>(p, inst, B, psi, o, ws, s, y, lam, active, stats);
    case 64: return dispatch_phi<DIM, 64>(p, inst, B, psi, o, ws, s, y, lam, active, stats);
    default: return dispatch_phi<DIM, 128>(p, inst, B, psi, o, ws, s, y, lam, active, stats);
  }
}

size_t problem_bytes(const sdf_problem *p) {
  if (p->csr) {
    const long long N = p->P.N, nnz = (long long)p->sci.size();
    size_t o = 0;
    o = al(o + sizeof(double) * N);        // inverse diagonal of S
    o = al(o + sizeof(float) * N);         // its FP32 copy
    o = al(o + sizeof(int) * (N + 1));     // S row pointers
    o = al(o + sizeof(int) * nnz);         // S column indices
    o = al(o + sizeof(double) * nnz);      // S values
    return o;
  }
  const auto &d = p->d;
  long long nx = d.n[0], ny = d.n[1], nz = d.dim == 3 ? d.n[2] : 1;
  long long N = nx * ny * nz;
  size_t o = 0;
  o = al(o + sizeof(double) * N);  // shared Jacobi diagonal
  o = al(o + sizeof(float) * N);   // its FP32 copy
  if (d.has_kappa) {
    o = al(o + sizeof(double) * N);                     // kappa
    o = al(o + sizeof(double) * (nx + 1) * ny * nz);    // fx
    o = al(o + sizeof(double) * nx * (ny + 1) * nz);    // fy
    if (d.dim == 3) o = al(o + sizeof(double) * nx * ny * (nz + 1));
    o = al(o + sizeof(float) * (nx + 1) * ny * nz);     // FP32 copies of fx, fy, fz
    o = al(o + sizeof(float) * nx * (ny + 1) * nz);
    if (d.dim == 3) o = al(o + sizeof(float) * nx * ny * (nz + 1));
  }
  return o;
}

}  // namespace

// Accessors for the eigensolver translation unit (not part of the C ABI).
const sdf::OpParams *sdf_internal_op(const sdf_problem *p, int *nsm, int *convection) {
  if (!p || !p->bound) return nullptr;
  if (nsm) *nsm = p->nsm;
  if (convection) *convection = p->P.convection;
  return &p->P;
}
void sdf_internal_set_error(sdf_problem *p, const char *msg) {
  if (p) p->err = msg;
}
const sdf_problem_desc *sdf_internal_desc(const sdf_problem *p, const double **kappa_host) {
  if (!p) return nullptr;
  if (kappa_host) *kappa_host = p->kappa.empty() ? nullptr : p->kappa.data();
  return &p->d;
}
// S_II (mode 0) or S (mode 1) applied to `cols` columns of N doubles at once
// (the restricted eigensolve's block), one launch
sdf_status sdf_internal_apply_S_cols(sdf_problem *p, const double *inst_dev,
                                     const uint8_t *active_dev, const double *u, double *out,
                                     int cols, int mode, cudaStream_t s) {
  if (cols < 1 || cols > 65535) return fail(p, SDF_ERR_INVALID_ARG, "bad column count");
  const OpParams &P = p->P;
  const int GX = std::max(1, p->nsm * 4 / cols);
  const dim3 g(GX, cols);
  if (P.dim == 1) k_apply<1><<<g, NT, 0, s>>>(P, inst_dev, active_dev, u, out, mode, GX);
  else if (P.dim == 2) k_apply<2><<<g, NT, 0, s>>>(P, inst_dev, active_dev, u, out, mode, GX);
  else k_apply<3><<<g, NT, 0, s>>>(P, inst_dev, active_dev, u, out, mode, GX);
  CKL("k_apply");
  p->prof.launches += 1;
  return SDF_OK;
}
// the registered reference modes (nullptr when none)
const void *sdf_internal_modes(const sdf_problem *p, int *k, long long *ld, sdf_dtype *dtype) {
  if (!p || !p->phi) return nullptr;
  *k = p->k;
  *ld = p->ld;
  *dtype = p->phi_dtype;
  return p->phi;
}

// ===========================================================================
// C ABI

extern "C" {

void sdf_default_opts(sdf_opts *o) {
  if (!o) return;
  o->rtol = 1e-8;
  o->tau = 1e-10;
  o->tau_cond = 1e10;
  o->max_outer = 30;
  o->max_cg = 1000000;
  o->deflate = 1;
  o->check_every = 64;
  o->profile = 0;
  o->max_blocks = 0;
  o->precision = SDF_PREC_F64;
  o->replace_every = 100;
  o->max_launches = 0;
  o->ritz_r = 0;
  o->safe_r = 0;
  o->tau_safe = 1e4;
  o->tau_dep = 1e-10;
  o->floor_c = 10.0;
  o->column_depth = 0;
  o->column_pairs = 0;
  o->graph = 1;
}

sdf_status sdf_problem_create(const sdf_problem_desc *desc, const double *kappa_host,
                              sdf_problem **out) {
  if (!desc || !out) return SDF_ERR_INVALID_ARG;
  *out = nullptr;
  const sdf_problem_desc &d = *desc;
  if (d.dim != 2 && d.dim != 3) return SDF_ERR_INVALID_ARG;
  for (int i = 0; i < d.dim; ++i)
    if (d.n[i] < 1 || d.n[i] > (1 << 20)) return SDF_ERR_INVALID_ARG;
  if (!(d.alpha > 0) || !(d.mass > 0) || !(d.kscale > 0) || !(d.diff_scale > 0) ||
      !(d.yd_sigma > 0))
    return SDF_ERR_INVALID_ARG;
  if (d.has_kappa && !kappa_host) return SDF_ERR_INVALID_ARG;
  if (d.time_axis && (d.dim != 3 || !(d.t_final > 0) || !(d.ramp_tau > 0)))
    return SDF_ERR_INVALID_ARG;
  long long nz = d.dim == 3 ? d.n[2] : 1;
  long long N = (long long)d.n[0] * d.n[1] * nz;
  if (N > (1LL << 31)) return SDF_ERR_INVALID_ARG;
  sdf_problem *p = new sdf_problem();
  p->d = d;
  if (d.has_kappa) {
    p->kappa.assign(kappa_host, kappa_host + N);
    for (double v : p->kappa)
      if (!(v > 0) || !std::isfinite(v)) {
        delete p;
        return SDF_ERR_INVALID_ARG;
      }
  }
  OpParams &P = p->P;
  memset(&P, 0, sizeof(P));
  P.dim = d.dim;
  P.nx = d.n[0];
  P.ny = d.n[1];
  P.nz = (int)nz;
  P.N = N;
  P.mass = d.mass;
  P.wgt = d.alpha * d.kscale * d.kscale / d.mass;
  int n3[3] = {P.nx, P.ny, P.nz};
  for (int i = 0; i < 3; ++i) {
    P.h[i] = i < d.dim ? 1.0 / (n3[i] + 1) : 1.0;
    P.inv_h[i] = i < d.dim ? (double)(n3[i] + 1) : 0.0;
    P.cdiff[i] = i < d.dim ? d.diff_scale * P.inv_h[i] * P.inv_h[i] : 0.0;
    P.cdf[i] = (float)P.cdiff[i];
  }
  P.massf = (float)P.mass;
  P.wgtf = (float)P.wgt;
  P.convection = d.convection;
  P.inst_conv = d.convection;
  P.yd_sigma = d.yd_sigma;
  if (d.time_axis) {
    // axis 2 is time: no diffusion along it, the implicit Euler difference
    // as an upwind term (the convection code path), dt = t_final / n_t
    P.time_axis = 1;
    P.convection = 1;
    P.dt = d.t_final / (double)nz;
    P.cb_t = 1.0 / P.dt;
    P.ramp_tau = d.ramp_tau;
    P.cdiff[2] = 0.0;
    P.cdf[2] = 0.0f;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      p->nsm = v;
  }
  if (cudaHostAlloc((void **)&p->pinned, 4 * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return SDF_ERR_CUDA;
  }
  p->ev_ready = true;
  for (int i = 0; i < 8; ++i)
    if (cudaEventCreate(&p->ev[i]) != cudaSuccess) p->ev_ready = false;
  cudaGetLastError();
  *out = p;
  return SDF_OK;
}

sdf_status sdf_problem_create_csr(int64_t n, const int32_t *rowptr, const int32_t *col,
                                  const double *val, double mass, double alpha, double kscale,
                                  sdf_problem **out) {
  if (!out) return SDF_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || n > (1LL << 30) || !rowptr || !col || !val || !(mass > 0) || !(alpha > 0) ||
      !(kscale > 0) || rowptr[0] != 0)
    return SDF_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return SDF_ERR_INVALID_ARG;
  const int64_t nnz = rowptr[n];
  for (int64_t q = 0; q < nnz; ++q)
    if (col[q] < 0 || col[q] >= n || !std::isfinite(val[q])) return SDF_ERR_INVALID_ARG;
  // K^T by rows (the columns of K), entries in increasing row order
  std::vector<int> tp(n + 1, 0), ti(nnz);
  std::vector<double> tv(nnz);
  for (int64_t q = 0; q < nnz; ++q) ++tp[col[q] + 1];
  for (int64_t i = 0; i < n; ++i) tp[i + 1] += tp[i];
  {
    std::vector<int> fill(tp.begin(), tp.end() - 1);
    for (int64_t r = 0; r < n; ++r)
      for (int q = rowptr[r]; q < rowptr[r + 1]; ++q) {
        const int a = fill[col[q]]++;
        ti[a] = (int)r;
        tv[a] = val[q];
      }
  }
  // S = mass I + wgt K^T K row by row (Gustavson): row i of K^T K is the sum
  // over the entries K_ri of K_ri times row r of K
  sdf_problem *p = new sdf_problem();
  p->csr = true;
  const double wgt = alpha * kscale * kscale / mass;
  p->srp.assign(n + 1, 0);
  p->sdinv.assign(n, 0.0);
  std::vector<int> mark(n, -1), cols;
  std::vector<double> acc(n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    cols.clear();
    mark[i] = (int)i;
    acc[i] = mass;
    cols.push_back((int)i);
    for (int a = tp[i]; a < tp[i + 1]; ++a) {
      const int r = ti[a];
      const double kri = tv[a];
      for (int q = rowptr[r]; q < rowptr[r + 1]; ++q) {
        const int j = col[q];
        if (mark[j] != (int)i) {
          mark[j] = (int)i;
          acc[j] = 0.0;
          cols.push_back(j);
        }
        acc[j] += wgt * kri * val[q];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int j : cols) {
      p->sci.push_back(j);
      p->sv.push_back(acc[j]);
    }
    p->srp[i + 1] = (int)p->sci.size();
    p->sdinv[i] = 1.0 / acc[i];
  }
  if (p->sci.size() > (size_t)INT_MAX) {
    delete p;
    return SDF_ERR_UNSUPPORTED;
  }
  // DIM = 1: the rows in tiles of 256 consecutive nodes
  sdf_problem_desc &d = p->d;
  memset(&d, 0, sizeof(d));
  d.dim = 1;
  d.n[0] = (int)n;
  d.n[1] = 1;
  d.n[2] = 1;
  d.alpha = alpha;
  d.mass = mass;
  d.kscale = kscale;
  d.diff_scale = 1.0;
  d.yd_sigma = 1.0;
  OpParams &P = p->P;
  memset(&P, 0, sizeof(P));
  P.dim = 1;
  P.nx = (int)n;
  P.ny = 1;
  P.nz = 1;
  P.N = n;
  P.mass = mass;
  P.wgt = wgt;
  P.massf = (float)mass;
  P.wgtf = (float)wgt;
  for (int i = 0; i < 3; ++i) {
    P.h[i] = 1.0;
    P.inv_h[i] = 1.0;
  }
  P.yd_sigma = 1.0;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      p->nsm = v;
  }
  if (cudaHostAlloc((void **)&p->pinned, 4 * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return SDF_ERR_CUDA;
  }
  p->ev_ready = true;
  for (int i = 0; i < 8; ++i)
    if (cudaEventCreate(&p->ev[i]) != cudaSuccess) p->ev_ready = false;
  cudaGetLastError();
  *out = p;
  return SDF_OK;
}

sdf_status sdf_solve_batch_rhs(sdf_problem *p, const double *inst_dev, const double *rhs_dev,
                               int batch, const double *psi_dev, const sdf_opts *opts, void *ws,
                               size_t ws_bytes, void *stream, double *y_dev, double *lambda_dev,
                               uint8_t *active_dev, sdf_stats *stats_host) {
  if (!p) return SDF_ERR_INVALID_ARG;
  if (!rhs_dev) return fail(p, SDF_ERR_INVALID_ARG, "NULL rhs");
  if (!inst_dev && p->P.inst_conv)
    return fail(p, SDF_ERR_INVALID_ARG, "the instances' convection velocities are needed");
  p->P.rhs = rhs_dev;
  sdf_status st = sdf_solve_batch(p, inst_dev, batch, psi_dev, opts, ws, ws_bytes, stream, y_dev,
                                  lambda_dev, active_dev, stats_host);
  p->P.rhs = nullptr;
  return st;
}

sdf_status sdf_problem_device_bytes(const sdf_problem *p, size_t *bytes) {
  if (!p || !bytes) return SDF_ERR_INVALID_ARG;
  *bytes = problem_bytes(p);
  return SDF_OK;
}

sdf_status sdf_problem_bind(sdf_problem *p, void *dev_buf, size_t bytes, void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  size_t need = problem_bytes(p);
  if (!dev_buf || !aligned(dev_buf, 256))
    return fail(p, SDF_ERR_INVALID_ARG, "problem buffer must be a 256-byte aligned device pointer");
  if (bytes < need) return fail(p, SDF_ERR_WORKSPACE, "problem buffer too small");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaGetDevice(&p->device));
  char *base = (char *)dev_buf;
  OpParams &P = p->P;
  size_t o = 0;
  p->dinv_shared = (double *)(base + o);
  o = al(o + sizeof(double) * P.N);
  p->dinv_shared32 = (float *)(base + o);
  o = al(o + sizeof(float) * P.N);
  P.fx = P.fy = P.fz = nullptr;
  P.fxf = P.fyf = P.fzf = nullptr;
  if (p->csr) {
    const long long nnz = (long long)p->sci.size();
    int *rp = (int *)(base + o);
    o = al(o + sizeof(int) * (P.N + 1));
    int *ci = (int *)(base + o);
    o = al(o + sizeof(int) * nnz);
    double *v = (double *)(base + o);
    std::vector<float> d32(p->sdinv.begin(), p->sdinv.end());
    CK(cudaMemcpyAsync(rp, p->srp.data(), sizeof(int) * (P.N + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ci, p->sci.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(v, p->sv.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->dinv_shared, p->sdinv.data(), sizeof(double) * P.N,
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->dinv_shared32, d32.data(), sizeof(float) * P.N, cudaMemcpyHostToDevice,
                       s));
    CK(cudaStreamSynchronize(s));  // the host copies are pageable and d32 is local
    P.csr_rp = rp;
    P.csr_ci = ci;
    P.csr_v = v;
    p->dev = dev_buf;
    p->dev_bytes = bytes;
    p->bound = true;
    return SDF_OK;
  }
  if (p->d.has_kappa) {
    double *kap = (double *)(base + o);
    o = al(o + sizeof(double) * P.N);
    double *fx = (double *)(base + o);
    o = al(o + sizeof(double) * (P.nx + 1) * (long long)P.ny * P.nz);
    double *fy = (double *)(base + o);
    o = al(o + sizeof(double) * P.nx * (long long)(P.ny + 1) * P.nz);
    double *fz = nullptr;
    if (P.dim == 3) {
      fz = (double *)(base + o);
      o = al(o + sizeof(double) * P.nx * (long long)P.ny * (P.nz + 1));
    }
    float *fxf = (float *)(base + o);
    o = al(o + sizeof(float) * (P.nx + 1) * (long long)P.ny * P.nz);
    float *fyf = (float *)(base + o);
    o = al(o + sizeof(float) * P.nx * (long long)(P.ny + 1) * P.nz);
    float *fzf = P.dim == 3 ? (float *)(base + o) : nullptr;
    CK(cudaMemcpyAsync(kap, p->kappa.data(), sizeof(double) * P.N, cudaMemcpyHostToDevice, s));
    k_faces<<<p->nsm * 4, NT, 0, s>>>(P, kap, p->d.diff_scale, fx, fy, fz, fxf, fyf, fzf);
    CKL("k_faces");
    P.fx = fx;
    P.fy = fy;
    P.fz = fz;
    P.fxf = fxf;
    P.fyf = fyf;
    P.fzf = fzf;
  }
  if (P.dim == 2) k_diag_shared<2><<<p->nsm * 4, NT, 0, s>>>(P, p->dinv_shared, p->dinv_shared32);
  else k_diag_shared<3><<<p->nsm * 4, NT, 0, s>>>(P, p->dinv_shared, p->dinv_shared32);
  CKL("k_diag_shared");
  CK(cudaStreamSynchronize(s));
  p->dev = dev_buf;
  p->dev_bytes = bytes;
  p->bound = true;
  return SDF_OK;
}

sdf_status sdf_set_reference_modes(sdf_problem *p, const void *phi_dev, int k, int64_t ld,
                                   sdf_dtype dtype) {
  if (!p) return SDF_ERR_INVALID_ARG;
  if (k < 1 || k > SDF_MAX_K) return fail(p, SDF_ERR_UNSUPPORTED, "k must be in [1, SDF_MAX_K]");
  if (!phi_dev || !aligned(phi_dev, 16))
    return fail(p, SDF_ERR_INVALID_ARG, "Phi must be a 16-byte aligned device pointer");
  if (ld < p->P.N) return fail(p, SDF_ERR_INVALID_ARG, "ld must be >= N");
  if (dtype != SDF_F64 && dtype != SDF_F32 && dtype != SDF_BF16)
    return fail(p, SDF_ERR_INVALID_ARG, "unknown dtype");
  p->phi = phi_dev;
  p->k = k;
  p->ld = ld;
  p->phi_dtype = dtype;
  return SDF_OK;
}

sdf_status sdf_analytic_modes(sdf_problem *p, int k, void *phi_dev, int64_t ld, sdf_dtype dtype,
                              double *eigvals_host, void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  if (!phi_dev || k < 1 || ld < p->P.N) return fail(p, SDF_ERR_INVALID_ARG, "bad arguments");
  if (k > SDF_MAX_K) return fail(p, SDF_ERR_UNSUPPORTED, "k > SDF_MAX_K");
  if (p->P.time_axis)
    return fail(p, SDF_ERR_UNSUPPORTED,
                "no closed-form modes on a space-time problem: build I_nt (x) Z_s with "
                "sdf_spacetime_kron_modes");
  if (p->csr) return fail(p, SDF_ERR_UNSUPPORTED, "no closed-form modes without a grid");
  const int dim = p->d.dim;
  int n[3] = {p->P.nx, p->P.ny, p->P.nz};
  // enumerate multi-indices with small eigenvalue sums; mu_q per direction
  int m[3] = {1, 1, 1};
  int lim = (int)std::ceil(std::pow(4.0 * k, 1.0 / dim)) + 4;
  for (int d = 0; d < dim; ++d) m[d] = std::min(n[d], lim);
  struct Cand {
    double lam;
    int i[3];
  };
  std::vector<Cand> c;
  for (int a = 1; a <= m[0]; ++a)
    for (int b = 1; b <= m[1]; ++b)
      for (int e = 1; e <= (dim == 3 ? m[2] : 1); ++e) {
        int ii[3] = {a, b, dim == 3 ? e : 1};
        double mu[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) {
          double h = 1.0 / (n[d] + 1);
          double sn = std::sin(ii[d] * M_PI / (2.0 * (n[d] + 1)));
          mu[d] = 4.0 / (h * h) * sn * sn;
        }
        std::sort(mu, mu + dim);  // order-independent sum: exact ties stay ties
        double sum = 0.0;
        for (int d = 0; d < dim; ++d) sum += mu[d];
        c.push_back({sum, {ii[0], ii[1], ii[2]}});
      }
  if ((int)c.size() < k) return fail(p, SDF_ERR_INVALID_ARG, "k larger than the grid supports");
  std::stable_sort(c.begin(), c.end(), [&](const Cand &x, const Cand &y) {
    if (x.lam != y.lam) return x.lam < y.lam;
    for (int d = dim - 1; d >= 0; --d)
      if (x.i[d] != y.i[d]) return x.i[d] < y.i[d];
    return false;
  });
  std::vector<int> idx(3 * k);
  for (int j = 0; j < k; ++j)
    for (int d = 0; d < 3; ++d) idx[3 * j + d] = c[j].i[d];
  if (eigvals_host) {
    double ds = p->d.diff_scale;
    for (int j = 0; j < k; ++j)
      eigvals_host[j] = p->P.mass + p->P.wgt * (ds * c[j].lam) * (ds * c[j].lam);
  }
  cudaStream_t s = (cudaStream_t)stream;
  ModeIdx tab;
  memset(&tab, 0, sizeof(tab));
  for (int j = 0; j < 3 * k; ++j) tab.v[j] = idx[j];
  const int grid = p->nsm * 8;
  switch (dtype) {
    case SDF_F64:
      k_sine_modes<double><<<grid, NT, 0, s>>>(dim, n[0], n[1], n[2], tab, k, (double *)phi_dev, ld);
      break;
    case SDF_F32:
      k_sine_modes<float><<<grid, NT, 0, s>>>(dim, n[0], n[1], n[2], tab, k, (float *)phi_dev, ld);
      break;
    case SDF_BF16:
      k_sine_modes<__nv_bfloat16><<<grid, NT, 0, s>>>(dim, n[0], n[1], n[2], tab, k,
                                                      (__nv_bfloat16 *)phi_dev, ld);
      break;
    default:
      return fail(p, SDF_ERR_INVALID_ARG, "unknown dtype");
  }
  CKL("k_sine_modes");
  p->prof.launches += 1;
  return SDF_OK;
}

sdf_status sdf_workspace_size(const sdf_problem *p, int batch, const sdf_opts *opts, size_t *bytes) {
  if (!p || !bytes || batch < 1) return SDF_ERR_INVALID_ARG;
  *bytes = make_layout(p, batch, opts ? opts->max_blocks : 0,
                       opts ? (opts->precision == SDF_PREC_MIXED) : 0).total;
  return SDF_OK;
}

sdf_status sdf_host_io_bytes(const sdf_problem *p, int batch, size_t *bytes) {
  if (!p || !bytes || batch < 1) return SDF_ERR_INVALID_ARG;
  long long N = p->P.N;
  *bytes = al(sizeof(double) * 7 * batch) + al(sizeof(double) * N) +
           2 * al(sizeof(double) * N * batch) + al((size_t)N * batch);
  return SDF_OK;
}

static sdf_status check_solve_args(sdf_problem *p, int batch, const sdf_opts *opts, void *ws,
                                   size_t ws_bytes) {
  if (!p) return SDF_ERR_INVALID_ARG;
  if (!p->bound) return fail(p, SDF_ERR_INVALID_ARG, "problem not bound (sdf_problem_bind)");
  if (batch < 1 || batch > 65535) return fail(p, SDF_ERR_INVALID_ARG, "batch out of range");
  if (!opts) return fail(p, SDF_ERR_INVALID_ARG, "opts is NULL");
  if (opts->max_outer < 1 || opts->max_outer > SDF_MAX_OUTER)
    return fail(p, SDF_ERR_INVALID_ARG, "max_outer must be in [1, SDF_MAX_OUTER]");
  if (opts->max_cg < 0 || !(opts->rtol >= 0) || opts->max_blocks < 0)
    return fail(p, SDF_ERR_INVALID_ARG, "bad opts");
  if (!ws || !aligned(ws, 256))
    return fail(p, SDF_ERR_INVALID_ARG, "workspace must be a 256-byte aligned device pointer");
  if (opts->precision != SDF_PREC_F64 && opts->precision != SDF_PREC_MIXED)
    return fail(p, SDF_ERR_INVALID_ARG, "unknown precision");
  if (opts->precision == SDF_PREC_MIXED && p->csr)
    return fail(p, SDF_ERR_UNSUPPORTED, "a problem given by its operator runs on the FP64 path");
  if (opts->precision == SDF_PREC_MIXED && p->P.convection)
    return fail(p, SDF_ERR_UNSUPPORTED,
                "the mixed path is not validated for convection (FP32 attainable accuracy above "
                "rtol stalls its refinement loop); use SDF_PREC_F64");
  if (opts->replace_every < 0) return fail(p, SDF_ERR_INVALID_ARG, "replace_every < 0");
  if (!(opts->floor_c >= 0.0)) return fail(p, SDF_ERR_INVALID_ARG, "floor_c < 0");
  {
    const int cd = opts->column_depth;
    if (cd != 0 && cd != 8 && cd != 16 && cd != 32 && cd != 64)
      return fail(p, SDF_ERR_INVALID_ARG, "column_depth must be 0, 8, 16, 32 or 64");
    if (opts->column_pairs < 0 || opts->column_pairs > 2)
      return fail(p, SDF_ERR_INVALID_ARG, "column_pairs must be 0, 1 or 2");
  }
  if (opts->precision == SDF_PREC_MIXED && p->P.N > 2147483647LL)
    return fail(p, SDF_ERR_UNSUPPORTED, "the mixed path indexes one instance with 32 bits");
  size_t need = make_layout(p, batch, opts->max_blocks, opts->precision == SDF_PREC_MIXED).total;
  if (ws_bytes < need) return fail(p, SDF_ERR_WORKSPACE, "workspace too small");
  return SDF_OK;
}

sdf_status sdf_solve_batch(sdf_problem *p, const double *inst_dev, int batch, const double *psi_dev,
                           const sdf_opts *opts, void *ws, size_t ws_bytes, void *stream,
                           double *y_dev, double *lambda_dev, uint8_t *active_dev,
                           sdf_stats *stats_host) {
  sdf_status st = check_solve_args(p, batch, opts, ws, ws_bytes);
  if (st != SDF_OK) return st;
  if ((!inst_dev && !p->P.rhs) || !psi_dev || !y_dev || !active_dev)
    return fail(p, SDF_ERR_INVALID_ARG, "NULL input or output pointer");
  if (p->csr && !p->P.rhs)
    return fail(p, SDF_ERR_INVALID_ARG,
                "a problem given by its operator has no desired state: use sdf_solve_batch_rhs");
  p->err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  if (p->d.dim == 1)
    return dispatch_k<1>(p, inst_dev, batch, psi_dev, *opts, (char *)ws, s, y_dev, lambda_dev,
                         active_dev, stats_host);
  if (p->d.dim == 2)
    return dispatch_k<2>(p, inst_dev, batch, psi_dev, *opts, (char *)ws, s, y_dev, lambda_dev,
                         active_dev, stats_host);
  return dispatch_k<3>(p, inst_dev, batch, psi_dev, *opts, (char *)ws, s, y_dev, lambda_dev,
                       active_dev, stats_host);
}

sdf_status sdf_solve_batch_x0(sdf_problem *p, const double *inst_dev, int batch,
                              const double *psi_dev, const double *x0_dev, const sdf_opts *opts,
                              void *ws, size_t ws_bytes, void *stream, double *y_dev,
                              double *lambda_dev, uint8_t *active_dev, sdf_stats *stats_host) {
  if (!p) return SDF_ERR_INVALID_ARG;
  if (!x0_dev) return fail(p, SDF_ERR_INVALID_ARG, "NULL x0");
  p->x0 = x0_dev;
  sdf_status st = sdf_solve_batch(p, inst_dev, batch, psi_dev, opts, ws, ws_bytes, stream, y_dev,
                                  lambda_dev, active_dev, stats_host);
  p->x0 = nullptr;
  return st;
}

sdf_status sdf_autotune(sdf_problem *p, const double *inst_dev, int batch, const double *psi_dev,
                        const sdf_opts *opts, void *ws, size_t ws_bytes, void *stream,
                        double *y_dev, uint8_t *active_dev, int *choice) {
  if (!p || !opts) return SDF_ERR_INVALID_ARG;
  sdf_status st = check_solve_args(p, batch, opts, ws, ws_bytes);
  if (st != SDF_OK) return st;
  if (!inst_dev || !psi_dev || !y_dev || !active_dev)
    return fail(p, SDF_ERR_INVALID_ARG, "NULL input or output pointer");
  int best = 0;
  if (p->d.dim == 3 && opts->precision == SDF_PREC_MIXED) {
    cudaStream_t s = (cudaStream_t)stream;
    sdf_opts o = *opts;
    o.max_cg = 40;  // a short, capped solve per candidate
    o.profile = 0;
    float best_ms = 0.0f;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    o.column_depth = 0;
    o.column_pairs = 0;
    int best_pairs = 0;
    for (int pr : {1, 2}) {  // instance pairs, then one instance per block
      if (pr == 1 && batch < 2) continue;
      for (int zc : {8, 16, 32, 64}) {
        p->force_zc = zc;
        p->force_pairs = pr;
        for (int rep = 0; rep < 2; ++rep) {  // the first run warms up
          CK(cudaEventRecord(e0, s));
          st = sdf_solve_batch(p, inst_dev, batch, psi_dev, &o, ws, ws_bytes, stream, y_dev,
                               nullptr, active_dev, nullptr);
          CK(cudaEventRecord(e1, s));
          CK(cudaEventSynchronize(e1));
          if (st != SDF_OK && st != SDF_ERR_CG_MAXIT) {
            p->force_zc = 0;
            p->force_pairs = 0;
            return st;
          }
        }
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (best == 0 || ms < best_ms) {
          best = zc;
          best_pairs = pr == 1 ? 1 : 0;
          best_ms = ms;
        }
      }
    }
    p->force_zc = 0;
    p->force_pairs = 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->tuned_zc[batch] = best;
    p->tuned_pairs[batch] = best_pairs;
  }
  if (choice) *choice = best;
  return SDF_OK;
}

sdf_status sdf_learned_host_io_bytes(const sdf_problem *p, const sdf_warm_model *M, int batch,
                                     size_t *bytes) {
  if (!p || !M || !bytes || batch < 1) return SDF_ERR_INVALID_ARG;
  size_t io = 0, pw = 0;
  if (sdf_host_io_bytes(p, batch, &io) != SDF_OK) return SDF_ERR_INVALID_ARG;
  if (sdf_warm_predict_workspace_size(M, batch, &pw) != SDF_OK)
    return fail((sdf_problem *)p, SDF_ERR_INVALID_ARG,
                std::string("warm-start model: ") + sdf_aux_last_error());
  *bytes = al(io) + al(sizeof(double) * (size_t)p->P.N * batch) + al(pw);
  return SDF_OK;
}

sdf_status sdf_solve_batch_learned_host(sdf_problem *p, const sdf_warm_model *M,
                                        const double *inst_host, int batch,
                                        const double *psi_host, const sdf_opts *opts, void *ws,
                                        size_t ws_bytes, void *stream, double *y_host,
                                        double *lambda_host, uint8_t *active_host,
                                        sdf_stats *stats_host) {
  if (!p) return SDF_ERR_INVALID_ARG;
  if (!M || !inst_host || !psi_host || !y_host || !active_host)
    return fail(p, SDF_ERR_INVALID_ARG, "NULL model or host pointer");
  if (M->n != p->P.N) return fail(p, SDF_ERR_INVALID_ARG, "warm-start model has another N");
  size_t need = 0, extra = 0, io = 0;
  if (batch < 1) return fail(p, SDF_ERR_INVALID_ARG, "batch out of range");
  sdf_status st = sdf_workspace_size(p, batch, opts, &need);
  if (st != SDF_OK) return st;
  st = sdf_learned_host_io_bytes(p, M, batch, &extra);
  if (st != SDF_OK) return st;
  sdf_host_io_bytes(p, batch, &io);
  if (ws_bytes < al(need) + extra) return fail(p, SDF_ERR_WORKSPACE, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = p->P.N;
  char *base = (char *)ws + al(need);
  double *inst_d = (double *)base;
  double *psi_d = (double *)(base + al(sizeof(double) * 7 * batch));
  double *y_d = (double *)((char *)psi_d + al(sizeof(double) * N));
  double *lam_d = (double *)((char *)y_d + al(sizeof(double) * N * batch));
  uint8_t *act_d = (uint8_t *)((char *)lam_d + al(sizeof(double) * N * batch));
  double *x0_d = (double *)(base + al(io));
  char *pws = (char *)x0_d + al(sizeof(double) * (size_t)N * batch);
  const size_t pws_bytes = ws_bytes - (size_t)(pws - (char *)ws);
  CK(cudaMemcpyAsync(inst_d, inst_host, sizeof(double) * 7 * batch, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(psi_d, psi_host, sizeof(double) * N, cudaMemcpyHostToDevice, s));
  st = sdf_warm_predict(M, inst_d, batch, x0_d, pws, pws_bytes, stream);
  if (st != SDF_OK) return fail(p, st, std::string("warm-start prediction: ") + sdf_aux_last_error());
  st = sdf_solve_batch_x0(p, inst_d, batch, psi_d, x0_d, opts, ws, need, stream, y_d,
                          lambda_host ? lam_d : nullptr, act_d, stats_host);
  if (st != SDF_OK && st != SDF_ERR_CG_MAXIT && st != SDF_ERR_OUTER_MAXIT &&
      st != SDF_ERR_BREAKDOWN && st != SDF_ERR_NONFINITE)
    return st;
  CK(cudaMemcpyAsync(y_host, y_d, sizeof(double) * N * batch, cudaMemcpyDeviceToHost, s));
  if (lambda_host)
    CK(cudaMemcpyAsync(lambda_host, lam_d, sizeof(double) * N * batch, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(active_host, act_d, (size_t)N * batch, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return st;
}

sdf_status sdf_autotune_choice(const sdf_problem *p, int batch, int *depth, int *pairs) {
  if (!p || !depth || !pairs) return SDF_ERR_INVALID_ARG;
  auto iz = p->tuned_zc.find(batch);
  auto ip = p->tuned_pairs.find(batch);
  *depth = iz == p->tuned_zc.end() ? 0 : iz->second;
  *pairs = ip == p->tuned_pairs.end() ? -1 : ip->second;
  return SDF_OK;
}

sdf_status sdf_solve_batch_host(sdf_problem *p, const double *inst_host, int batch,
                                const double *psi_host, const sdf_opts *opts, void *ws,
                                size_t ws_bytes, void *stream, double *y_host, double *lambda_host,
                                uint8_t *active_host, sdf_stats *stats_host) {
  if (!p) return SDF_ERR_INVALID_ARG;
  if (!inst_host || !psi_host || !y_host || !active_host)
    return fail(p, SDF_ERR_INVALID_ARG, "NULL host pointer");
  size_t need = 0, io = 0;
  if (batch < 1) return fail(p, SDF_ERR_INVALID_ARG, "batch out of range");
  sdf_workspace_size(p, batch, opts, &need);
  sdf_host_io_bytes(p, batch, &io);
  if (ws_bytes < need + io) return fail(p, SDF_ERR_WORKSPACE, "workspace too small for host I/O");
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = p->P.N;
  char *base = (char *)ws + al(need);
  double *inst_d = (double *)base;
  base += al(sizeof(double) * 7 * batch);
  double *psi_d = (double *)base;
  base += al(sizeof(double) * N);
  double *y_d = (double *)base;
  base += al(sizeof(double) * N * batch);
  double *lam_d = (double *)base;
  base += al(sizeof(double) * N * batch);
  uint8_t *act_d = (uint8_t *)base;
  if (ws_bytes < al(need) + io) return fail(p, SDF_ERR_WORKSPACE, "workspace too small for host I/O");
  CK(cudaMemcpyAsync(inst_d, inst_host, sizeof(double) * 7 * batch, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(psi_d, psi_host, sizeof(double) * N, cudaMemcpyHostToDevice, s));
  sdf_status st = sdf_solve_batch(p, inst_d, batch, psi_d, opts, ws, need, stream, y_d,
                                  lambda_host ? lam_d : nullptr, act_d, stats_host);
  if (st != SDF_OK && st != SDF_ERR_CG_MAXIT && st != SDF_ERR_OUTER_MAXIT &&
      st != SDF_ERR_BREAKDOWN && st != SDF_ERR_NONFINITE)
    return st;
  CK(cudaMemcpyAsync(y_host, y_d, sizeof(double) * N * batch, cudaMemcpyDeviceToHost, s));
  if (lambda_host)
    CK(cudaMemcpyAsync(lambda_host, lam_d, sizeof(double) * N * batch, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(active_host, act_d, (size_t)N * batch, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return st;
}

sdf_status sdf_spacetime_kron_modes(sdf_problem *p, const void *zs_dev, int r, int64_t ldz,
                                    sdf_dtype dtype, void *phi_dev, int64_t ld, void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  if (!p->P.time_axis) return fail(p, SDF_ERR_INVALID_ARG, "not a space-time problem");
  const long long Ns = (long long)p->P.nx * p->P.ny;
  const int nt = p->P.nz;
  if (!zs_dev || !phi_dev || r < 1 || ldz < Ns || ld < p->P.N)
    return fail(p, SDF_ERR_INVALID_ARG, "bad arguments");
  if ((long long)r * nt > SDF_MAX_K) return fail(p, SDF_ERR_UNSUPPORTED, "r n_t > SDF_MAX_K");
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned g = (unsigned)p->nsm * 8;
  if (dtype == SDF_F64)
    k_kron_time<double><<<g, NT, 0, s>>>((const double *)zs_dev, ldz, r, Ns, nt, (double *)phi_dev, ld);
  else if (dtype == SDF_F32)
    k_kron_time<float><<<g, NT, 0, s>>>((const float *)zs_dev, ldz, r, Ns, nt, (float *)phi_dev, ld);
  else if (dtype == SDF_BF16)
    k_kron_time<__nv_bfloat16><<<g, NT, 0, s>>>((const __nv_bfloat16 *)zs_dev, ldz, r, Ns, nt,
                                                 (__nv_bfloat16 *)phi_dev, ld);
  else
    return fail(p, SDF_ERR_INVALID_ARG, "unknown dtype");
  CKL("k_kron_time");
  p->prof.launches += 1;
  return SDF_OK;
}

void sdf_dct2_basis(int n, int r, double *w_host) {
  if (!w_host || n < 1 || r < 1 || r > n) return;
  const double pi = 3.14159265358979323846;
  for (int a = 0; a < r; ++a)
    for (int l = 0; l < n; ++l)
      w_host[l + (size_t)a * n] =
          std::sqrt((a == 0 ? 1.0 : 2.0) / n) * std::cos(pi * (l + 0.5) * a / n);
}

sdf_status sdf_spacetime_modes(sdf_problem *p, const double *wt_host, int rt, const void *zs_dev,
                               int r, int64_t ldz, sdf_dtype dtype, void *phi_dev, int64_t ld,
                               void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  if (!p->P.time_axis) return fail(p, SDF_ERR_INVALID_ARG, "not a space-time problem");
  const long long Ns = (long long)p->P.nx * p->P.ny;
  const int nt = p->P.nz;
  if (!wt_host || !zs_dev || !phi_dev || r < 1 || rt < 1 || ldz < Ns || ld < p->P.N)
    return fail(p, SDF_ERR_INVALID_ARG, "bad arguments");
  if ((long long)nt * rt > SDF_TB_MAX)
    return fail(p, SDF_ERR_UNSUPPORTED, "n_t r_t above 1024");
  if ((long long)r * rt > SDF_MAX_K) return fail(p, SDF_ERR_UNSUPPORTED, "r r_t > SDF_MAX_K");
  TemporalBasis tb{};
  tb.nt = nt;
  tb.rt = rt;
  for (long long e = 0; e < (long long)nt * rt; ++e) tb.w[e] = wt_host[e];
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned g = (unsigned)p->nsm * 8;
  if (dtype == SDF_F64)
    k_time_basis<double><<<g, NT, 0, s>>>(tb, (const double *)zs_dev, ldz, r, Ns, (double *)phi_dev, ld);
  else if (dtype == SDF_F32)
    k_time_basis<float><<<g, NT, 0, s>>>(tb, (const float *)zs_dev, ldz, r, Ns, (float *)phi_dev, ld);
  else if (dtype == SDF_BF16)
    k_time_basis<__nv_bfloat16><<<g, NT, 0, s>>>(tb, (const __nv_bfloat16 *)zs_dev, ldz, r, Ns,
                                                  (__nv_bfloat16 *)phi_dev, ld);
  else
    return fail(p, SDF_ERR_INVALID_ARG, "unknown dtype");
  CKL("k_time_basis");
  p->prof.launches += 1;
  return SDF_OK;
}

sdf_status sdf_apply_S(sdf_problem *p, const double *inst_dev, const uint8_t *active_dev,
                       const double *u_dev, double *out_dev, int mode, void *ws, size_t ws_bytes,
                       void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  if (!p->bound) return fail(p, SDF_ERR_INVALID_ARG, "problem not bound");
  if (!inst_dev || !u_dev || !out_dev || (mode == 0 && !active_dev) || (mode != 0 && mode != 1))
    return fail(p, SDF_ERR_INVALID_ARG, "bad arguments");
  (void)ws;
  (void)ws_bytes;
  cudaStream_t s = (cudaStream_t)stream;
  const OpParams &P = p->P;
  int GX = p->nsm * 4;
  if (P.dim == 1) k_apply<1><<<GX, NT, 0, s>>>(P, inst_dev, active_dev, u_dev, out_dev, mode, GX);
  else if (P.dim == 2)
    k_apply<2><<<GX, NT, 0, s>>>(P, inst_dev, active_dev, u_dev, out_dev, mode, GX);
  else k_apply<3><<<GX, NT, 0, s>>>(P, inst_dev, active_dev, u_dev, out_dev, mode, GX);
  CKL("k_apply");
  p->prof.launches += 1;
  return SDF_OK;
}

sdf_status sdf_project(sdf_problem *p, const uint8_t *active_dev, const double *v_dev,
                       double *out_dev, void *ws, size_t ws_bytes, void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  if (!p->phi) return fail(p, SDF_ERR_INVALID_ARG, "no reference modes registered");
  if (p->phi_dtype != SDF_F64) return fail(p, SDF_ERR_UNSUPPORTED, "FP64 modes expected");
  if (!active_dev || !v_dev || !out_dev) return fail(p, SDF_ERR_INVALID_ARG, "NULL pointer");
  int GX = p->nsm * 2;
  int KM = kmax_for(p->k);
  size_t need = al(sizeof(double) * (size_t)GX * KM) + al(sizeof(int) * NCNT);
  if (!ws || !aligned(ws, 256) || ws_bytes < need)
    return fail(p, SDF_ERR_WORKSPACE, "workspace too small for sdf_project");
  double *part = (double *)ws;
  int *cnt = (int *)((char *)ws + al(sizeof(double) * (size_t)GX * KM));
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemsetAsync(cnt, 0, sizeof(int) * NCNT, s));
  const double *Phi = (const double *)p->phi;
  dim3 g(1, GX);
  switch (KM) {
    case 16: k_project<16, double><<<g, NT, 0, s>>>(Phi, p->ld, p->k, p->P.N, active_dev, v_dev, nullptr, out_dev, part, cnt, GX); break;
    case 32: k_project<32, double><<<g, NT, 0, s>>>(Phi, p->ld, p->k, p->P.N, active_dev, v_dev, nullptr, out_dev, part, cnt, GX); break;
    case 64: k_project<64, double><<<g, NT, 0, s>>>(Phi, p->ld, p->k, p->P.N, active_dev, v_dev, nullptr, out_dev, part, cnt, GX); break;
    default: k_project<128, double><<<g, NT, 0, s>>>(Phi, p->ld, p->k, p->P.N, active_dev, v_dev, nullptr, out_dev, part, cnt, GX); break;
  }
  CKL("k_project");
  p->prof.launches += 1;
  return SDF_OK;
}

// ---------------------------------------------------------------------------
// sdf_project_noalloc: sdf_project with its scratch in a fixed device array.
// The array holds the per-block partial sums (SDF_NOALLOC_BLOCKS blocks x
// SDF_MAX_K modes, as doubles) followed by the last-block ticket counters.
// It is shared by every call on a device and lives as long as the library.

#define SDF_NOALLOC_BLOCKS 512
#define SDF_NOALLOC_DOUBLES (SDF_NOALLOC_BLOCKS * SDF_MAX_K + 64)

static __device__ __align__(256) double g_noalloc_scratch[SDF_NOALLOC_DOUBLES];

// Device address of g_noalloc_scratch, looked up once per device (the symbol
// name is only a host-side stand-in; kernels need the real device address).
static double *g_noalloc_addr[64];
static std::mutex g_noalloc_mu;

static sdf_status noalloc_scratch(sdf_problem *p, double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_check(p, e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(p, SDF_ERR_UNSUPPORTED, "device index >= 64");
  // the scratch address is per device: the problem's data (and the modes the
  // kernel reads) live on the device it was bound on
  if (p->device >= 0 && dev != p->device)
    return fail(p, SDF_ERR_INVALID_ARG,
                "sdf_project_noalloc: the current device is not the one the problem was bound on");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_check(p, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_addr[dev] = (double *)ptr;
  }
  *out = g_noalloc_addr[dev];
  return SDF_OK;
}

sdf_status sdf_project_noalloc(sdf_problem *p, const uint8_t *active_dev, const double *v_dev,
                               double *out_dev, void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  if (!p->phi) return fail(p, SDF_ERR_INVALID_ARG, "no reference modes registered");
  if (p->phi_dtype != SDF_F64) return fail(p, SDF_ERR_UNSUPPORTED, "FP64 modes expected");
  if (!active_dev || !v_dev || !out_dev) return fail(p, SDF_ERR_INVALID_ARG, "NULL pointer");
  if (p->k < 1 || p->k > SDF_MAX_K)
    return fail(p, SDF_ERR_UNSUPPORTED,
                "sdf_project_noalloc: k exceeds the static scratch limit SDF_MAX_K (128)");
  const int KM = kmax_for(p->k);
  const int GX = std::min(p->nsm * 2, SDF_NOALLOC_BLOCKS);
  if ((size_t)GX * KM + NCNT > (size_t)SDF_NOALLOC_DOUBLES)
    return fail(p, SDF_ERR_UNSUPPORTED, "sdf_project_noalloc: scratch limit exceeded");
  double *scratch = nullptr;
  sdf_status st = noalloc_scratch(p, &scratch);
  if (st != SDF_OK) return st;
  double *part = scratch;
  int *cnt = (int *)(scratch + (size_t)SDF_NOALLOC_BLOCKS * SDF_MAX_K);
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemsetAsync(cnt, 0, sizeof(int) * NCNT, s));  // tickets must start at zero
  const double *Phi = (const double *)p->phi;
  dim3 g(1, GX);
  switch (KM) {
    case 16: k_project<16, double><<<g, NT, 0, s>>>(Phi, p->ld, p->k, p->P.N, active_dev, v_dev, nullptr, out_dev, part, cnt, GX); break;
    case 32: k_project<32, double><<<g, NT, 0, s>>>(Phi, p->ld, p->k, p->P.N, active_dev, v_dev, nullptr, out_dev, part, cnt, GX); break;
    case 64: k_project<64, double><<<g, NT, 0, s>>>(Phi, p->ld, p->k, p->P.N, active_dev, v_dev, nullptr, out_dev, part, cnt, GX); break;
    default: k_project<128, double><<<g, NT, 0, s>>>(Phi, p->ld, p->k, p->P.N, active_dev, v_dev, nullptr, out_dev, part, cnt, GX); break;
  }
  CKL("k_project (static scratch)");
  p->prof.launches += 1;
  return SDF_OK;
}

sdf_status sdf_get_profile(const sdf_problem *p, sdf_profile *out) {
  if (!p || !out) return SDF_ERR_INVALID_ARG;
  *out = p->prof;
  return SDF_OK;
}

sdf_status sdf_reset_profile(sdf_problem *p) {
  if (!p) return SDF_ERR_INVALID_ARG;
  memset(&p->prof, 0, sizeof(p->prof));
  return SDF_OK;
}

const char *sdf_last_error(const sdf_problem *p) { return p ? p->err.c_str() : "null handle"; }

void sdf_problem_destroy(sdf_problem *p) {
  if (!p) return;
  if (p->pinned) cudaFreeHost(p->pinned);
  for (int i = 0; i < 8; ++i)
    if (p->ev[i]) cudaEventDestroy(p->ev[i]);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  delete p;
}

}  // extern "C"
