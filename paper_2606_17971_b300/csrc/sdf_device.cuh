// sdf_device.cuh -- device-side building blocks of the sm_103a solver:
// the matrix-free masked application of S = mass I + w A^T A (flux form,
// halo-2 shared-memory tiles), projections onto the reference modes, and the
// deterministic grid reductions.  Included only by sdf.cu.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/sdf.h"

namespace sdf {

constexpr int NT = 256;          // threads per block of every tile kernel
constexpr int NWARP = NT / 32;

// --------------------------------------------------------------------------
// Operator description passed by value to kernels.
struct OpParams {
  int dim, nx, ny, nz;
  long long N;
  double mass, wgt;        // S = mass I + wgt A^T A, wgt = alpha kscale^2 / mass
  double cdiff[3];         // diff_scale / h_d^2 for kappa = 1
  double inv_h[3];
  const double *fx, *fy, *fz;  // face coefficients (already scaled) or null
  int convection;
  double yd_sigma;
  double h[3];
  // FP32 copies for the FP32 stencils of the mixed path: read straight from
  // the parameter bank, never converted per use (a conversion issues on the
  // FP64 pipe, 1/64 of the FP32 rate on this part)
  float cdf[3], massf, wgtf;
  const float *fxf, *fyf, *fzf;  // face coefficients in FP32 or null
  // space-time problems (App. E.2): axis 2 is time, the backward difference
  // (u_l - u_{l-1}) / dt enters A as an upwind term of coefficient
  // cb_t = 1 / dt; y_d carries the ramp 1 - exp(-t / ramp_tau)
  int time_axis;
  double cb_t, dt, ramp_tau;
  int inst_conv;  // instances' convection velocities are applied (in space)
  // a problem given by its operator K (sdf_problem_create_csr): S assembled
  // as CSR (rows of the pseudo-grid's nodes), applied row by row
  const int *csr_rp, *csr_ci;
  const double *csr_v;
  // caller-given right-hand sides (instance-major, stride N) in place of
  // mass y_d, for sdf_solve_batch_rhs; null otherwise
  const double *rhs;
};

// Operator constants and face arrays in arithmetic type T.
template <class T> struct OpT;
template <> struct OpT<double> {
  static __device__ __forceinline__ double cd(const OpParams &P, int d) { return P.cdiff[d]; }
  static __device__ __forceinline__ double mass(const OpParams &P) { return P.mass; }
  static __device__ __forceinline__ double wgt(const OpParams &P) { return P.wgt; }
  static __device__ __forceinline__ const double *fx(const OpParams &P) { return P.fx; }
  static __device__ __forceinline__ const double *fy(const OpParams &P) { return P.fy; }
  static __device__ __forceinline__ const double *fz(const OpParams &P) { return P.fz; }
};
template <> struct OpT<float> {
  static __device__ __forceinline__ float cd(const OpParams &P, int d) { return P.cdf[d]; }
  static __device__ __forceinline__ float mass(const OpParams &P) { return P.massf; }
  static __device__ __forceinline__ float wgt(const OpParams &P) { return P.wgtf; }
  static __device__ __forceinline__ const float *fx(const OpParams &P) { return P.fxf; }
  static __device__ __forceinline__ const float *fy(const OpParams &P) { return P.fyf; }
  static __device__ __forceinline__ const float *fz(const OpParams &P) { return P.fzf; }
};

// Tile shapes: 2D 64 x 8 (halo 2 in x, y), 3D 32 x 4 x 4 (halo 2 everywhere).
template <int DIM> struct TileCfg;
template <> struct TileCfg<2> {
  static constexpr int TX = 64, TY = 8, TZ = 1, HZ = 0, HZ1 = 0;
};
template <> struct TileCfg<3> {
  static constexpr int TX = 32, TY = 4, TZ = 4, HZ = 2, HZ1 = 1;
};
// DIM = 1: a problem given by its operator (CSR S), tiles of 256 rows
template <> struct TileCfg<1> {
  static constexpr int TX = 256, TY = 1, TZ = 1, HZ = 0, HZ1 = 0;
};

// Shared-memory tile of the stencil in arithmetic type T (double for the FP64
// path, float for the FP32 part of the mixed path).
template <int DIM, class T = double> struct TileSmem {
  using C = TileCfg<DIM>;
  static constexpr int UX = C::TX + 4, UY = C::TY + 4, UZ = C::TZ + 2 * C::HZ;
  static constexpr int WX = C::TX + 2, WY = C::TY + 2, WZ = C::TZ + 2 * C::HZ1;
  static constexpr int TILE = C::TX * C::TY * C::TZ;
  T u[UZ * UY * UX];
  T w[WZ * WY * WX];
  T v[TILE];
};
// the CSR tiles keep only the tile-local output vector
template <class T> struct TileSmem<1, T> {
  static constexpr int TILE = TileCfg<1>::TX;
  T v[TILE];
};

template <int DIM>
__device__ __forceinline__ int uidx(int lx, int ly, int lz) {
  using S = TileSmem<DIM, double>;
  return (lx + 2) + S::UX * ((ly + 2) + S::UY * (lz + TileCfg<DIM>::HZ));
}
template <int DIM>
__device__ __forceinline__ int widx(int lx, int ly, int lz) {
  using S = TileSmem<DIM, double>;
  return (lx + 1) + S::WX * ((ly + 1) + S::WY * (lz + TileCfg<DIM>::HZ1));
}

// Face coefficients in arithmetic type T: constant-kappa problems use the
// per-kernel constant cd[d]; variable kappa reads the array of type T.
template <class T>
__device__ __forceinline__ T fx_T(const OpParams &P, const T cd[3], int i, int j, int l) {
  const T *f = OpT<T>::fx(P);
  return f ? __ldg(f + i + (long long)(P.nx + 1) * (j + (long long)P.ny * l)) : cd[0];
}
template <class T>
__device__ __forceinline__ T fy_T(const OpParams &P, const T cd[3], int i, int j, int l) {
  const T *f = OpT<T>::fy(P);
  return f ? __ldg(f + i + (long long)P.nx * (j + (long long)(P.ny + 1) * l)) : cd[1];
}
template <class T>
__device__ __forceinline__ T fz_T(const OpParams &P, const T cd[3], int i, int j, int l) {
  const T *f = OpT<T>::fz(P);
  return f ? __ldg(f + i + (long long)P.nx * (j + (long long)P.ny * l)) : cd[2];
}

__device__ __forceinline__ double face_x(const OpParams &P, int i, int j, int l) {
  return P.fx ? __ldg(P.fx + i + (long long)(P.nx + 1) * (j + (long long)P.ny * l)) : P.cdiff[0];
}
__device__ __forceinline__ double face_y(const OpParams &P, int i, int j, int l) {
  return P.fy ? __ldg(P.fy + i + (long long)P.nx * (j + (long long)(P.ny + 1) * l)) : P.cdiff[1];
}
__device__ __forceinline__ double face_z(const OpParams &P, int i, int j, int l) {
  return P.fz ? __ldg(P.fz + i + (long long)P.nx * (j + (long long)P.ny * l)) : P.cdiff[2];
}

// (A u)_p in flux form: sum over faces of k_f (u_p - u_nb) plus first-order
// upwind convection; U(dx,dy,dz) returns u at the offset (0 outside the grid).
template <int DIM, class T, class U>
__device__ __forceinline__ T apply_A(const OpParams &P, const T cb[3], const T cd[3], int i,
                                     int j, int l, U u) {
  T c = u(0, 0, 0);
  T s = fx_T(P, cd, i, j, l) * (c - u(-1, 0, 0)) + fx_T(P, cd, i + 1, j, l) * (c - u(1, 0, 0));
  s += fy_T(P, cd, i, j, l) * (c - u(0, -1, 0)) + fy_T(P, cd, i, j + 1, l) * (c - u(0, 1, 0));
  if (DIM == 3)
    s += fz_T(P, cd, i, j, l) * (c - u(0, 0, -1)) + fz_T(P, cd, i, j, l + 1) * (c - u(0, 0, 1));
  if (cb[0] > (T)0) s += cb[0] * (c - u(-1, 0, 0));
  else if (cb[0] < (T)0) s -= cb[0] * (c - u(1, 0, 0));
  if (cb[1] > (T)0) s += cb[1] * (c - u(0, -1, 0));
  else if (cb[1] < (T)0) s -= cb[1] * (c - u(0, 1, 0));
  if (DIM == 3) {
    if (cb[2] > (T)0) s += cb[2] * (c - u(0, 0, -1));
    else if (cb[2] < (T)0) s -= cb[2] * (c - u(0, 0, 1));
  }
  return s;
}

// (A^T w)_p: the diffusion part is symmetric; the upwind part is transposed
// (a backward difference becomes a forward one and vice versa).
template <int DIM, class T, class U>
__device__ __forceinline__ T apply_AT(const OpParams &P, const T cb[3], const T cd[3], int i,
                                      int j, int l, U w) {
  T c = w(0, 0, 0);
  T s = fx_T(P, cd, i, j, l) * (c - w(-1, 0, 0)) + fx_T(P, cd, i + 1, j, l) * (c - w(1, 0, 0));
  s += fy_T(P, cd, i, j, l) * (c - w(0, -1, 0)) + fy_T(P, cd, i, j + 1, l) * (c - w(0, 1, 0));
  if (DIM == 3)
    s += fz_T(P, cd, i, j, l) * (c - w(0, 0, -1)) + fz_T(P, cd, i, j, l + 1) * (c - w(0, 0, 1));
  if (cb[0] > (T)0) s += cb[0] * (c - w(1, 0, 0));
  else if (cb[0] < (T)0) s -= cb[0] * (c - w(-1, 0, 0));
  if (cb[1] > (T)0) s += cb[1] * (c - w(0, 1, 0));
  else if (cb[1] < (T)0) s -= cb[1] * (c - w(0, -1, 0));
  if (DIM == 3) {
    if (cb[2] > (T)0) s += cb[2] * (c - w(0, 0, 1));
    else if (cb[2] < (T)0) s -= cb[2] * (c - w(0, 0, -1));
  }
  return s;
}

// Diagonal of S at node p: mass + wgt (A_pp^2 + sum over grid neighbours q of A_qp^2).
template <int DIM>
__device__ double diag_S(const OpParams &P, const double cb[3], int i, int j, int l) {
  int n[3] = {P.nx, P.ny, P.nz};
  int c[3] = {i, j, l};
  double app = 0.0, sq = 0.0;
  for (int d = 0; d < DIM; ++d) {
    double fw, fe;
    if (d == 0) { fw = face_x(P, i, j, l); fe = face_x(P, i + 1, j, l); }
    else if (d == 1) { fw = face_y(P, i, j, l); fe = face_y(P, i, j + 1, l); }
    else { fw = face_z(P, i, j, l); fe = face_z(P, i, j, l + 1); }
    double b = cb[d];
    app += fw + fe + fabs(b);
    if (c[d] - 1 >= 0) { double a = -fw - (b < 0.0 ? -b : 0.0); sq += a * a; }
    if (c[d] + 1 < n[d]) { double a = -fe - (b > 0.0 ? b : 0.0); sq += a * a; }
  }
  return P.mass + P.wgt * (app * app + sq);
}

// Tile origin of tile t.
template <int DIM>
__device__ __forceinline__ void tile_origin(const OpParams &P, long long t, int &ox, int &oy, int &oz) {
  using C = TileCfg<DIM>;
  int ntx = (P.nx + C::TX - 1) / C::TX, nty = (P.ny + C::TY - 1) / C::TY;
  ox = (int)(t % ntx) * C::TX;
  long long r = t / ntx;
  oy = (int)(r % nty) * C::TY;
  oz = (int)(r / nty) * C::TZ;
}

template <int DIM>
__host__ __device__ inline long long num_tiles(int nx, int ny, int nz) {
  using C = TileCfg<DIM>;
  return (long long)((nx + C::TX - 1) / C::TX) * ((ny + C::TY - 1) / C::TY) *
         ((nz + C::TZ - 1) / C::TZ);
}

// Apply S to the tile with origin (ox,oy,oz): load(gx,gy,gz,g) gives u at a grid
// node; store(e, gx, gy, gz, g, Su) receives S u at each grid node of the tile
// (e = local tile index).  Two shared-memory passes: w = A u on the halo-1
// ring, then mass u + wgt A^T w on the tile.  Work is mapped by x-rows: each
// warp takes whole rows and its lanes the x index, so the row's coordinates,
// global base index and bounds are computed once per row, and shared-memory
// neighbours are fixed offsets from the row base.
template <int DIM, class T, bool VARK, bool CONV, class Load, class Store>
__device__ __forceinline__ void tile_S_rows(const OpParams &P, const T cb[3], const T cd[3], T mass,
                                            T wgt, int ox, int oy, int oz, TileSmem<DIM, T> &sm,
                                            Load &load, Store &store) {
  using C = TileCfg<DIM>;
  using SM = TileSmem<DIM, T>;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const long long nxy = (long long)P.nx * P.ny;
  // phase 1: u on the halo-2 box, rows (ly, lz) of UX elements
  for (int row = warp; row < SM::UY * SM::UZ; row += NWARP) {
    const int ly = row % SM::UY - 2, lz = row / SM::UY - C::HZ;
    const int gy = oy + ly, gz = oz + lz;
    const bool rin = gy >= 0 && gy < P.ny && gz >= 0 && gz < P.nz;
    const long long g0 = (long long)gy * P.nx + gz * nxy + ox - 2;
    T *urow = sm.u + row * SM::UX;
    for (int lx = lane; lx < SM::UX; lx += 32) {
      const int gx = ox - 2 + lx;
      urow[lx] = (rin && gx >= 0 && gx < P.nx) ? (T)load(gx, gy, gz, g0 + lx) : (T)0;
    }
  }
  __syncthreads();
  // phase 2: w = A u on the halo-1 ring (zero outside the grid)
  constexpr int DU_X = 1, DU_Y = SM::UX, DU_Z = SM::UX * SM::UY;
  for (int row = warp; row < SM::WY * SM::WZ; row += NWARP) {
    const int ly = row % SM::WY - 1, lz = row / SM::WY - C::HZ1;
    const int gy = oy + ly, gz = oz + lz;
    const bool rin = gy >= 0 && gy < P.ny && gz >= 0 && gz < P.nz;
    const T *ubase = sm.u + (ly + 2) * SM::UX + (lz + C::HZ) * DU_Z + 2;  // u at (lx = 0)
    T *wrow = sm.w + row * SM::WX;
    for (int wx = lane; wx < SM::WX; wx += 32) {
      const int lx = wx - 1, gx = ox + lx;
      T val = (T)0;
      if (rin && gx >= 0 && gx < P.nx) {
        const T *uc = ubase + lx;
        const T c = uc[0];
        T fw, fe, fs, fn, fb = 0, ft = 0;
        if (VARK) {
          fw = fx_T(P, cd, gx, gy, gz); fe = fx_T(P, cd, gx + 1, gy, gz);
          fs = fy_T(P, cd, gx, gy, gz); fn = fy_T(P, cd, gx, gy + 1, gz);
          if (DIM == 3) { fb = fz_T(P, cd, gx, gy, gz); ft = fz_T(P, cd, gx, gy, gz + 1); }
        } else {
          fw = fe = cd[0]; fs = fn = cd[1];
          if (DIM == 3) fb = ft = cd[2];
        }
        const T um = uc[-DU_X], up = uc[DU_X], vm = uc[-DU_Y], vp = uc[DU_Y];
        T sacc = fw * (c - um) + fe * (c - up) + fs * (c - vm) + fn * (c - vp);
        T zm = 0, zp = 0;
        if (DIM == 3) {
          zm = uc[-DU_Z];
          zp = uc[DU_Z];
          sacc += fb * (c - zm) + ft * (c - zp);
        }
        if constexpr (CONV) {
          if (cb[0] > (T)0) sacc += cb[0] * (c - um);
          else if (cb[0] < (T)0) sacc -= cb[0] * (c - up);
          if (cb[1] > (T)0) sacc += cb[1] * (c - vm);
          else if (cb[1] < (T)0) sacc -= cb[1] * (c - vp);
          if (DIM == 3) {
            if (cb[2] > (T)0) sacc += cb[2] * (c - zm);
            else if (cb[2] < (T)0) sacc -= cb[2] * (c - zp);
          }
        }
        val = sacc;
      }
      wrow[wx] = val;
    }
  }
  __syncthreads();
  // phase 3: mass u + wgt A^T w on the tile
  constexpr int DW_X = 1, DW_Y = SM::WX, DW_Z = SM::WX * SM::WY;
  for (int row = warp; row < C::TY * C::TZ; row += NWARP) {
    const int ly = row % C::TY, lz = row / C::TY;
    const int gy = oy + ly, gz = oz + lz;
    const bool rin = gy < P.ny && gz < P.nz;
    const long long g0 = (long long)gy * P.nx + gz * nxy + ox;
    const T *wbase = sm.w + (ly + 1) * SM::WX + (lz + C::HZ1) * DW_Z + 1;
    const T *ubase = sm.u + (ly + 2) * SM::UX + (lz + C::HZ) * DU_Z + 2;
    for (int lx = lane; lx < C::TX; lx += 32) {
      const int e = lx + C::TX * row;
      const int gx = ox + lx;
      if (!rin || gx >= P.nx) {
        sm.v[e] = (T)0;
        continue;
      }
      const T *wc = wbase + lx;
      const T c = wc[0];
      T fw, fe, fs, fn, fb = 0, ft = 0;
      if (VARK) {
        fw = fx_T(P, cd, gx, gy, gz); fe = fx_T(P, cd, gx + 1, gy, gz);
        fs = fy_T(P, cd, gx, gy, gz); fn = fy_T(P, cd, gx, gy + 1, gz);
        if (DIM == 3) { fb = fz_T(P, cd, gx, gy, gz); ft = fz_T(P, cd, gx, gy, gz + 1); }
      } else {
        fw = fe = cd[0]; fs = fn = cd[1];
        if (DIM == 3) fb = ft = cd[2];
      }
      const T wm = wc[-DW_X], wp = wc[DW_X], vm = wc[-DW_Y], vp = wc[DW_Y];
      T sacc = fw * (c - wm) + fe * (c - wp) + fs * (c - vm) + fn * (c - vp);
      T zm = 0, zp = 0;
      if (DIM == 3) {
        zm = wc[-DW_Z];
        zp = wc[DW_Z];
        sacc += fb * (c - zm) + ft * (c - zp);
      }
      if constexpr (CONV) {  // transposed upwind part
        if (cb[0] > (T)0) sacc += cb[0] * (c - wp);
        else if (cb[0] < (T)0) sacc -= cb[0] * (c - wm);
        if (cb[1] > (T)0) sacc += cb[1] * (c - vp);
        else if (cb[1] < (T)0) sacc -= cb[1] * (c - vm);
        if (DIM == 3) {
          if (cb[2] > (T)0) sacc += cb[2] * (c - zp);
          else if (cb[2] < (T)0) sacc -= cb[2] * (c - zm);
        }
      }
      store(e, gx, gy, gz, g0 + lx, mass * ubase[lx] + wgt * sacc);
    }
  }
  __syncthreads();
}

// S u on the rows of a DIM = 1 tile from the assembled CSR S (a problem
// created from its operator K): one thread per row, the row's entries in
// order.  Out-of-range slots of sm.v are zeroed, as the stencil does.
template <int DIM, class T, class Load, class Store>
__device__ __forceinline__ void tile_S_csr(const OpParams &P, int ox, int oy, int oz,
                                           TileSmem<DIM, T> &sm, Load &load, Store &store) {
  using C = TileCfg<DIM>;
  constexpr int TILE = C::TX * C::TY * C::TZ;
  for (int e = threadIdx.x; e < TILE; e += blockDim.x) {
    const int lx = e % C::TX, row = e / C::TX, ly = row % C::TY, lz = row / C::TY;
    const int gx = ox + lx, gy = oy + ly, gz = oz + lz;
    if (gx >= P.nx || gy >= P.ny || gz >= P.nz) {
      sm.v[e] = (T)0;
      continue;
    }
    const long long g = gx + (long long)P.nx * (gy + (long long)P.ny * gz);
    double acc = 0.0;
    for (int q = P.csr_rp[g], qe = P.csr_rp[g + 1]; q < qe; ++q) {
      const int j = P.csr_ci[q];
      acc = fma(P.csr_v[q], (double)load(0, 0, 0, (long long)j), acc);
    }
    store(e, gx, gy, gz, g, (T)acc);
  }
  __syncthreads();
}

template <int DIM, class T, class Load, class Store>
__device__ __forceinline__ void tile_S_grid(const OpParams &P, const double cb64[3], int ox,
                                            int oy, int oz, TileSmem<DIM, T> &sm, Load &load,
                                            Store &store) {
  const T cb[3] = {(T)cb64[0], (T)cb64[1], (T)cb64[2]};
  const T cd[3] = {OpT<T>::cd(P, 0), OpT<T>::cd(P, 1), OpT<T>::cd(P, 2)};
  const T mass = OpT<T>::mass(P), wgt = OpT<T>::wgt(P);
  // the upwind terms are compiled only for problems with convection (their
  // per-point compares cost as much as the stencil on the FP64 pipe)
  if (P.convection) {
    if (P.fx)
      tile_S_rows<DIM, T, true, true>(P, cb, cd, mass, wgt, ox, oy, oz, sm, load, store);
    else
      tile_S_rows<DIM, T, false, true>(P, cb, cd, mass, wgt, ox, oy, oz, sm, load, store);
  } else {
    if (P.fx)
      tile_S_rows<DIM, T, true, false>(P, cb, cd, mass, wgt, ox, oy, oz, sm, load, store);
    else
      tile_S_rows<DIM, T, false, false>(P, cb, cd, mass, wgt, ox, oy, oz, sm, load, store);
  }
}

// S u on the tile with origin (ox, oy, oz): the row-wise CSR product on a
// problem given by its operator (DIM = 1), the stencil otherwise.
template <int DIM, class T, class Load, class Store>
__device__ void tile_S(const OpParams &P, const double cb64[3], int ox, int oy, int oz,
                       TileSmem<DIM, T> &sm, Load load, Store store) {
  if constexpr (DIM == 1) {
    tile_S_csr<DIM, T>(P, ox, oy, oz, sm, load, store);
  } else {
    tile_S_grid<DIM, T>(P, cb64, ox, oy, oz, sm, load, store);
  }
}

// ---------------------------------------------------------------------------
// 3D column stencil (2.5D blocking): an xy tile of CX x CY = 32 x 16 nodes
// marches in z through [z0, z1); each thread owns two output nodes.  Shared
// memory holds a ring of five u planes (z-2 .. z+2, halo 2 in x and y) and a
// ring of three w = A u planes (z-1 .. z+1, halo 1), so each node's u is
// loaded 36*20/512 = 1.4 times and its w computed 34*18/512 = 1.2 times.
// Ring slots rotate in registers.  Global loads run ahead of their use: the
// raw source values of plane z+3 and the output operands of plane z+1 are
// requested while plane z computes, and consumed one step later.
constexpr int CX = 32, CY = 16;
constexpr int CUX = CX + 4, CUY = CY + 4, CWX = CX + 2, CWY = CY + 2;
constexpr int CNU = CUX * CUY, CNW = CWX * CWY, CNO = CX * CY;
constexpr int CSU = (CNU + NT - 1) / NT, CSW = (CNW + NT - 1) / NT, CSO = CNO / NT;
static_assert(CNO % NT == 0, "whole output slots per thread");

// NA = 1: a second ring of five planes carries an auxiliary value of each u
// node (Src::AUX), read back at the output nodes; NA = 0 reserves nothing.
template <class T, int NA = 0> struct ColSmem {
  T u[5][CNU];
  T w[3][CNW];
  T a[NA ? 5 : 1][NA ? CNU : 1];
};

// Src: `Raw fetch(g)` issues the global loads of u at grid node g (index
// within the instance, 32-bit) and `T value(const Raw &)` turns them into u;
// with Src::AUX, `T aux(const Raw &)` is kept beside u.  Out: `Pre fetch(g)`
// loads the per-node operands of the output at g, and `store(g, Su, u_g,
// aux_g, pre)` receives S u.  CONV = false drops the upwind terms.
template <class T, bool VARK, bool CONV, class Src, class Out, int NA>
__device__ __forceinline__ void col_S3_impl(const OpParams &P, const T cb[3], const T cd[3], T mass,
                                            T wgt, int x0, int y0, int z0, int z1,
                                            ColSmem<T, NA> &sm, const Src &src, Out &out) {
  using Raw = typename Src::Raw;
  using Pre = typename Out::Pre;
  constexpr bool AUX = Src::AUX;
  static_assert(!AUX || NA == 1, "auxiliary ring");
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  // node indices within one instance fit in 32 bits (checked by the host)
  const int nxy = nx * ny, base = y0 * nx + x0;
  // u slots: shared index (-1: idle), in-grid flag, xy offset from the tile origin
  int ue[CSU], uoff[CSU];
  bool uok[CSU];
#pragma unroll
  for (int q = 0; q < CSU; ++q) {
    const int e = threadIdx.x + q * NT;
    const int lx = e % CUX - 2, ly = e / CUX - 2;
    ue[q] = e < CNU ? e : -1;
    uok[q] = e < CNU && x0 + lx >= 0 && x0 + lx < nx && y0 + ly >= 0 && y0 + ly < ny;
    uoff[q] = ly * nx + lx;
  }
  // w slots: shared index, centre in the u plane, in-grid flag
  int we[CSW], wuc[CSW];
  bool wok[CSW];
#pragma unroll
  for (int q = 0; q < CSW; ++q) {
    const int e = threadIdx.x + q * NT;
    const int lx = e % CWX - 1, ly = e / CWX - 1;
    we[q] = e < CNW ? e : -1;
    wok[q] = e < CNW && x0 + lx >= 0 && x0 + lx < nx && y0 + ly >= 0 && y0 + ly < ny;
    wuc[q] = (ly + 2) * CUX + (lx + 2);
  }
  // output slots
  int owc[CSO], ouc[CSO], ooff[CSO];
  bool ook[CSO];
#pragma unroll
  for (int q = 0; q < CSO; ++q) {
    const int e = threadIdx.x + q * NT;
    const int lx = e % CX, ly = e / CX;
    ook[q] = x0 + lx < nx && y0 + ly < ny;
    owc[q] = (ly + 1) * CWX + (lx + 1);
    ouc[q] = (ly + 2) * CUX + (lx + 2);
    ooff[q] = ly * nx + lx;
  }

  auto fetch = [&](int z, Raw (&raw)[CSU]) {
    const bool zin = z >= 0 && z < nz;
    const int zb = z * nxy + base;
#pragma unroll
    for (int q = 0; q < CSU; ++q) raw[q] = (zin && uok[q]) ? src.fetch(zb + uoff[q]) : Raw{};
  };
  auto put = [&](int z, int slot, const Raw (&raw)[CSU]) {
    const bool zin = z >= 0 && z < nz;
    T *up = sm.u[slot];
#pragma unroll
    for (int q = 0; q < CSU; ++q)
      if (ue[q] >= 0) {
        const bool on = zin && uok[q];
        up[ue[q]] = on ? src.value(raw[q]) : (T)0;
        if constexpr (AUX) sm.a[slot][ue[q]] = on ? src.aux(raw[q]) : (T)0;
      }
  };
  auto prefetch = [&](int z, Pre (&pr)[CSO]) {
    const int zb = z * nxy + base;
#pragma unroll
    for (int q = 0; q < CSO; ++q) pr[q] = ook[q] ? out.fetch(zb + ooff[q]) : Pre{};
  };
  // w = A u at plane z into slot ws, from u slots sm1, s0, sp1 (planes z-1, z, z+1)
  auto comp_w = [&](int z, int ws, int sm1, int s0, int sp1) {
    T *wp = sm.w[ws];
    const T *um = sm.u[sm1], *uc = sm.u[s0], *upl = sm.u[sp1];
    const bool zin = z >= 0 && z < nz;
#pragma unroll
    for (int q = 0; q < CSW; ++q) {
      if (we[q] < 0) continue;
      T val = (T)0;
      if (zin && wok[q]) {
        const int c0 = wuc[q];
        const T c = uc[c0];
        const T xm = uc[c0 - 1], xp = uc[c0 + 1], ym = uc[c0 - CUX], yp = uc[c0 + CUX];
        const T zm = um[c0], zp = upl[c0];
        T fw, fe, fs, fn, fb, ft;
        if (VARK) {
          const int gx = x0 + we[q] % CWX - 1, gy = y0 + we[q] / CWX - 1;
          fw = fx_T(P, cd, gx, gy, z); fe = fx_T(P, cd, gx + 1, gy, z);
          fs = fy_T(P, cd, gx, gy, z); fn = fy_T(P, cd, gx, gy + 1, z);
          fb = fz_T(P, cd, gx, gy, z); ft = fz_T(P, cd, gx, gy, z + 1);
        } else {
          fw = fe = cd[0]; fs = fn = cd[1]; fb = ft = cd[2];
        }
        T acc = fw * (c - xm) + fe * (c - xp) + fs * (c - ym) + fn * (c - yp) + fb * (c - zm) +
                ft * (c - zp);
        if (CONV) {
          if (cb[0] > (T)0) acc += cb[0] * (c - xm);
          else if (cb[0] < (T)0) acc -= cb[0] * (c - xp);
          if (cb[1] > (T)0) acc += cb[1] * (c - ym);
          else if (cb[1] < (T)0) acc -= cb[1] * (c - yp);
          if (cb[2] > (T)0) acc += cb[2] * (c - zm);
          else if (cb[2] < (T)0) acc -= cb[2] * (c - zp);
        }
        val = acc;
      }
      wp[we[q]] = val;
    }
  };
  // S u = mass u + wgt A^T w at plane z
  auto outputs = [&](int z, int wsm, int ws0, int wsp, int us0, const Pre (&pr)[CSO]) {
    const T *wm = sm.w[wsm], *wc = sm.w[ws0], *wpl = sm.w[wsp], *uc = sm.u[us0];
    const int zb = z * nxy + base;
#pragma unroll
    for (int q = 0; q < CSO; ++q) {
      if (!ook[q]) continue;
      const int o = owc[q];
      const T c = wc[o];
      const T xm = wc[o - 1], xp = wc[o + 1], ym = wc[o - CWX], yp = wc[o + CWX];
      const T zm = wm[o], zp = wpl[o];
      T fw, fe, fs, fn, fb, ft;
      if (VARK) {
        const int e = threadIdx.x + q * NT;
        const int gx = x0 + e % CX, gy = y0 + e / CX;
        fw = fx_T(P, cd, gx, gy, z); fe = fx_T(P, cd, gx + 1, gy, z);
        fs = fy_T(P, cd, gx, gy, z); fn = fy_T(P, cd, gx, gy + 1, z);
        fb = fz_T(P, cd, gx, gy, z); ft = fz_T(P, cd, gx, gy, z + 1);
      } else {
        fw = fe = cd[0]; fs = fn = cd[1]; fb = ft = cd[2];
      }
      T acc = fw * (c - xm) + fe * (c - xp) + fs * (c - ym) + fn * (c - yp) + fb * (c - zm) +
              ft * (c - zp);
      if (CONV) {
        if (cb[0] > (T)0) acc += cb[0] * (c - xp);
        else if (cb[0] < (T)0) acc -= cb[0] * (c - xm);
        if (cb[1] > (T)0) acc += cb[1] * (c - yp);
        else if (cb[1] < (T)0) acc -= cb[1] * (c - ym);
        if (cb[2] > (T)0) acc += cb[2] * (c - zp);
        else if (cb[2] < (T)0) acc -= cb[2] * (c - zm);
      }
      const T u0 = uc[ouc[q]];
      T ax = (T)0;
      if constexpr (AUX) ax = sm.a[us0][ouc[q]];
      out.store(zb + ooff[q], mass * u0 + wgt * acc, u0, ax, pr[q]);
    }
  };

  // ring slots of u planes z-2 .. z+2 and of w planes z-1 .. z+1
  int s0 = 0, s1 = 1, s2 = 2, s3 = 3, s4 = 4, t0 = 0, t1 = 1, t2 = 2;
  {  // prologue: u planes z0-2 .. z0+1 requested together
    Raw a[CSU], b[CSU], c[CSU], d[CSU];
    fetch(z0 - 2, a);
    fetch(z0 - 1, b);
    fetch(z0, c);
    fetch(z0 + 1, d);
    put(z0 - 2, 0, a);
    put(z0 - 1, 1, b);
    put(z0, 2, c);
    put(z0 + 1, 3, d);
  }
  Raw nxt[CSU];
  Pre pc[CSO], pn[CSO];
  fetch(z0 + 2, nxt);
  prefetch(z0, pc);
  __syncthreads();
  comp_w(z0 - 1, 0, 0, 1, 2);
  comp_w(z0, 1, 1, 2, 3);
  for (int z = z0; z < z1; ++z) {
    put(z + 2, s4, nxt);
    if (z + 1 < z1) {
      fetch(z + 3, nxt);
      prefetch(z + 1, pn);
    }
    __syncthreads();
    comp_w(z + 1, t2, s2, s3, s4);
    __syncthreads();
    outputs(z, t0, t1, t2, s2, pc);
    const int s = s0;
    s0 = s1; s1 = s2; s2 = s3; s3 = s4; s4 = s;
    const int t = t0;
    t0 = t1; t1 = t2; t2 = t;
#pragma unroll
    for (int q = 0; q < CSO; ++q) pc[q] = pn[q];
  }
  __syncthreads();
}

// Entry of the column stencil for kernels compiled per coefficient kind
// (VARK: face coefficients from kappa; CONV: upwind convection present).
template <class T, bool VARK, bool CONV, class Src, class Out, int NA>
__device__ __forceinline__ void col_S3(const OpParams &P, const double cb64[3], int x0, int y0,
                                       int z0, int z1, ColSmem<T, NA> &sm, const Src &src,
                                       Out &out) {
  const T cb[3] = {(T)cb64[0], (T)cb64[1], (T)cb64[2]};
  const T cd[3] = {OpT<T>::cd(P, 0), OpT<T>::cd(P, 1), OpT<T>::cd(P, 2)};
  col_S3_impl<T, VARK, CONV>(P, cb, cd, OpT<T>::mass(P), OpT<T>::wgt(P), x0, y0, z0, z1, sm, src,
                             out);
}

// ---------------------------------------------------------------------------
// Instance pairs: the same column stencil for two instances of a batch at
// once.  Both share the grid, so every slot index, bound and shared-memory
// offset is computed once for the pair; shared memory holds (instance 0,
// instance 1) pairs, so one 8-byte access moves both; and the arithmetic runs
// on packed FP32 pairs (add / sub / mul / fma .f32x2 of this part), each
// instruction doing the work of two scalar ones.
struct F2 {
  float x, y;
};
__device__ __forceinline__ F2 bc2(float a) { return F2{a, a}; }
__device__ __forceinline__ unsigned long long pk2(F2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ F2 upk2(unsigned long long r) {
  F2 o;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
  return o;
}
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(r);
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(r);
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(r);
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {  // a * b + c, one rounding
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
  return upk2(r);
}

// Compensated FP32 sums of a pair, as KahanF per half.
struct KahanF2 {
  F2 s{0.0f, 0.0f}, c{0.0f, 0.0f};
  __device__ __forceinline__ void add(F2 v) {
    const F2 y = sub2(v, c);
    const F2 t = add2(s, y);
    c = sub2(sub2(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value0() const { return (double)s.x - (double)c.x; }
  __device__ __forceinline__ double value1() const { return (double)s.y - (double)c.y; }
};

struct ColSmemPair {
  float2 u[5][CNU];
  float2 w[3][CNW];
};

// One side of the two-level stencil at a ring node: the sum over the six faces
// of f_face (c - nb), as two independent chains (lower and upper faces) added
// at the end, which halves the dependent-FMA latency of the scalar order.
__device__ __forceinline__ F2 flux6(F2 c, F2 xm, F2 xp, F2 ym, F2 yp, F2 zm, F2 zp, float fw,
                                   float fe, float fs, float fn, float fb, float ft) {
  F2 lo = mul2(bc2(fw), sub2(c, xm));
  F2 hi = mul2(bc2(fe), sub2(c, xp));
  lo = fma2(bc2(fs), sub2(c, ym), lo);
  hi = fma2(bc2(fn), sub2(c, yp), hi);
  lo = fma2(bc2(fb), sub2(c, zm), lo);
  hi = fma2(bc2(ft), sub2(c, zp), hi);
  return add2(lo, hi);
}

// Src: `Raw fetch(g)` issues the loads of both instances' u at node g and
// `F2 value(const Raw &)` forms the pair; Out: `Pre fetch(g)` and
// `store(g, Su, u_g, pre)` as in col_S3_impl, on pairs.  No convection (the
// mixed path refuses it), so the upwind terms are absent.  PF: the output
// operands are loaded one plane ahead (registers for latency); without it they
// are loaded at the output step (fewer registers, more resident blocks).
template <bool VARK, bool PF = true, class Src, class Out>
__device__ __forceinline__ void col_S3_pair(const OpParams &P, int x0, int y0, int z0, int z1,
                                            ColSmemPair &sm, const Src &src, Out &out) {
  using Raw = typename Src::Raw;
  using Pre = typename Out::Pre;
  const float cd[3] = {P.cdf[0], P.cdf[1], P.cdf[2]};
  const F2 mass = bc2(P.massf), wgt = bc2(P.wgtf);
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const int nxy = nx * ny, base = y0 * nx + x0;
  int ue[CSU], uoff[CSU];
  bool uok[CSU];
#pragma unroll
  for (int q = 0; q < CSU; ++q) {
    const int e = threadIdx.x + q * NT;
    const int lx = e % CUX - 2, ly = e / CUX - 2;
    ue[q] = e < CNU ? e : -1;
    uok[q] = e < CNU && x0 + lx >= 0 && x0 + lx < nx && y0 + ly >= 0 && y0 + ly < ny;
    uoff[q] = ly * nx + lx;
  }
  int we[CSW], wuc[CSW];
  bool wok[CSW];
#pragma unroll
  for (int q = 0; q < CSW; ++q) {
    const int e = threadIdx.x + q * NT;
    const int lx = e % CWX - 1, ly = e / CWX - 1;
    we[q] = e < CNW ? e : -1;
    wok[q] = e < CNW && x0 + lx >= 0 && x0 + lx < nx && y0 + ly >= 0 && y0 + ly < ny;
    wuc[q] = (ly + 2) * CUX + (lx + 2);
  }
  int owc[CSO], ouc[CSO], ooff[CSO];
  bool ook[CSO];
#pragma unroll
  for (int q = 0; q < CSO; ++q) {
    const int e = threadIdx.x + q * NT;
    const int lx = e % CX, ly = e / CX;
    ook[q] = x0 + lx < nx && y0 + ly < ny;
    owc[q] = (ly + 1) * CWX + (lx + 1);
    ouc[q] = (ly + 2) * CUX + (lx + 2);
    ooff[q] = ly * nx + lx;
  }
  auto ld2 = [](const float2 *a, int i) { const float2 v = a[i]; return F2{v.x, v.y}; };
  auto fetch = [&](int z, Raw (&raw)[CSU]) {
    const bool zin = z >= 0 && z < nz;
    const int zb = z * nxy + base;
#pragma unroll
    for (int q = 0; q < CSU; ++q) raw[q] = (zin && uok[q]) ? src.fetch(zb + uoff[q]) : Raw{};
  };
  auto put = [&](int z, int slot, const Raw (&raw)[CSU]) {
    const bool zin = z >= 0 && z < nz;
    float2 *up = sm.u[slot];
#pragma unroll
    for (int q = 0; q < CSU; ++q)
      if (ue[q] >= 0) {
        const F2 v = (zin && uok[q]) ? src.value(raw[q]) : F2{0.0f, 0.0f};
        up[ue[q]] = make_float2(v.x, v.y);
      }
  };
  auto prefetch = [&](int z, Pre (&pr)[CSO]) {
    const int zb = z * nxy + base;
#pragma unroll
    for (int q = 0; q < CSO; ++q) pr[q] = ook[q] ? out.fetch(zb + ooff[q]) : Pre{};
  };
  auto comp_w = [&](int z, int ws, int sm1, int s0, int sp1) {
    float2 *wp = sm.w[ws];
    const float2 *um = sm.u[sm1], *uc = sm.u[s0], *upl = sm.u[sp1];
    const bool zin = z >= 0 && z < nz;
#pragma unroll
    for (int q = 0; q < CSW; ++q) {
      if (we[q] < 0) continue;
      F2 val{0.0f, 0.0f};
      if (zin && wok[q]) {
        const int c0 = wuc[q];
        float fw, fe, fs, fn, fb, ft;
        if (VARK) {
          const int gx = x0 + we[q] % CWX - 1, gy = y0 + we[q] / CWX - 1;
          fw = fx_T<float>(P, cd, gx, gy, z); fe = fx_T<float>(P, cd, gx + 1, gy, z);
          fs = fy_T<float>(P, cd, gx, gy, z); fn = fy_T<float>(P, cd, gx, gy + 1, z);
          fb = fz_T<float>(P, cd, gx, gy, z); ft = fz_T<float>(P, cd, gx, gy, z + 1);
        } else {
          fw = fe = cd[0]; fs = fn = cd[1]; fb = ft = cd[2];
        }
        val = flux6(ld2(uc, c0), ld2(uc, c0 - 1), ld2(uc, c0 + 1), ld2(uc, c0 - CUX),
                    ld2(uc, c0 + CUX), ld2(um, c0), ld2(upl, c0), fw, fe, fs, fn, fb, ft);
      }
      wp[we[q]] = make_float2(val.x, val.y);
    }
  };
  auto outputs = [&](int z, int wsm, int ws0, int wsp, int us0, const Pre (&pr)[CSO]) {
    const float2 *wm = sm.w[wsm], *wc = sm.w[ws0], *wpl = sm.w[wsp], *uc = sm.u[us0];
    const int zb = z * nxy + base;
#pragma unroll
    for (int q = 0; q < CSO; ++q) {
      if (!ook[q]) continue;
      const int o = owc[q];
      float fw, fe, fs, fn, fb, ft;
      if (VARK) {
        const int e = threadIdx.x + q * NT;
        const int gx = x0 + e % CX, gy = y0 + e / CX;
        fw = fx_T<float>(P, cd, gx, gy, z); fe = fx_T<float>(P, cd, gx + 1, gy, z);
        fs = fy_T<float>(P, cd, gx, gy, z); fn = fy_T<float>(P, cd, gx, gy + 1, z);
        fb = fz_T<float>(P, cd, gx, gy, z); ft = fz_T<float>(P, cd, gx, gy, z + 1);
      } else {
        fw = fe = cd[0]; fs = fn = cd[1]; fb = ft = cd[2];
      }
      const F2 acc = flux6(ld2(wc, o), ld2(wc, o - 1), ld2(wc, o + 1), ld2(wc, o - CWX),
                           ld2(wc, o + CWX), ld2(wm, o), ld2(wpl, o), fw, fe, fs, fn, fb, ft);
      const F2 u0 = ld2(uc, ouc[q]);
      if constexpr (PF) {
        out.store(zb + ooff[q], fma2(wgt, acc, mul2(mass, u0)), u0, pr[q]);
      } else {
        const Pre now = out.fetch(zb + ooff[q]);
        out.store(zb + ooff[q], fma2(wgt, acc, mul2(mass, u0)), u0, now);
      }
    }
  };
  int s0 = 0, s1 = 1, s2 = 2, s3 = 3, s4 = 4, t0 = 0, t1 = 1, t2 = 2;
  {
    Raw a[CSU], b[CSU], c[CSU], d[CSU];
    fetch(z0 - 2, a);
    fetch(z0 - 1, b);
    fetch(z0, c);
    fetch(z0 + 1, d);
    put(z0 - 2, 0, a);
    put(z0 - 1, 1, b);
    put(z0, 2, c);
    put(z0 + 1, 3, d);
  }
  Raw nxt[CSU];
  Pre pc[PF ? CSO : 1], pn[PF ? CSO : 1];
  fetch(z0 + 2, nxt);
  if constexpr (PF) prefetch(z0, pc);
  __syncthreads();
  comp_w(z0 - 1, 0, 0, 1, 2);
  comp_w(z0, 1, 1, 2, 3);
  for (int z = z0; z < z1; ++z) {
    put(z + 2, s4, nxt);
    if (z + 1 < z1) {
      fetch(z + 3, nxt);
      if constexpr (PF) prefetch(z + 1, pn);
    }
    __syncthreads();
    comp_w(z + 1, t2, s2, s3, s4);
    __syncthreads();
    if constexpr (PF) {
      outputs(z, t0, t1, t2, s2, pc);
    } else {
      Pre none[CSO];
      outputs(z, t0, t1, t2, s2, none);
    }
    const int s = s0;
    s0 = s1; s1 = s2; s2 = s3; s3 = s4; s4 = s;
    const int t = t0;
    t0 = t1; t1 = t2; t2 = t;
    if constexpr (PF) {
#pragma unroll
      for (int q = 0; q < CSO; ++q) pc[q] = pn[q];
    }
  }
  __syncthreads();
}

// Column work items of a 3D grid: xy tiles x z-chunks of zc planes.
__host__ __device__ inline long long col_items(int nx, int ny, int nz, int zc) {
  return (long long)((nx + CX - 1) / CX) * ((ny + CY - 1) / CY) * ((nz + zc - 1) / zc);
}
__device__ __forceinline__ void col_origin(const OpParams &P, long long t, int zc, int &x0, int &y0,
                                           int &z0, int &z1) {
  int ntx = (P.nx + CX - 1) / CX, nty = (P.ny + CY - 1) / CY;
  x0 = (int)(t % ntx) * CX;
  long long r = t / ntx;
  y0 = (int)(r % nty) * CY;
  z0 = (int)(r / nty) * zc;
  z1 = min(z0 + zc, P.nz);
}

// Accumulate acc[jj] += sum over the tile of Phi_j(g) v(g) for modes
// j = warp + NWARP*jj < k; lanes run over the contiguous x-rows of the tile
// (coalesced reads of each mode).  v is the tile-local vector in shared memory
// (zero outside I and outside the grid).
template <int DIM, int KMAX, class PhiT, class T>
__device__ __forceinline__ void tile_project(const OpParams &P, const PhiT *__restrict__ Phi,
                                             long long ld, int k, int ox, int oy, int oz,
                                             const T *v_s, double (&acc)[KMAX / NWARP]) {
  using C = TileCfg<DIM>;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
  for (int jj = 0; jj < KMAX / NWARP; ++jj) {
    int j = warp + NWARP * jj;
    if (j < k) {
      const PhiT *ph = Phi + (long long)j * ld;
      T s = (T)0;
      for (int e = lane; e < C::TX * C::TY * C::TZ; e += 32) {
        int lx = e % C::TX;
        int t = e / C::TX;
        int gx = ox + lx, gy = oy + t % C::TY, gz = oz + t / C::TY;
        if (gx < P.nx && gy < P.ny && gz < P.nz) {
          long long g = gx + (long long)P.nx * (gy + (long long)P.ny * gz);
          s = fma((T)ph[g], v_s[e], s);
        }
      }
      acc[jj] += (double)s;
    }
  }
}

// Compensated (Kahan) FP32 accumulator: FP32 adds with the rounding error
// carried along, converted to FP64 once per thread.
struct KahanF {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of one double (all threads get the result).
__device__ __forceinline__ double block_sum(double v, double *red /* NWARP doubles */) {
  v = warp_sum(v);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < NWARP; ++w) s += red[w];
  __syncthreads();
  return s;
}

// Block reduction of per-thread mode accumulators: out[j] = sum over the
// block's threads of acc[j], j < k (FP32 per thread, FP64 across threads).
// scratch: NT doubles of shared memory.
template <int KMAX>
__device__ __forceinline__ void block_sum_modes(const float (&acc)[KMAX], int k, double *out,
                                                double *scratch) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
  for (int j0 = 0; j0 < KMAX; j0 += 32) {
    // lane l of each warp ends with the warp's sum for mode j0 + l
    double mine = 0.0;
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      double v = (j0 + l < KMAX) ? (double)acc[j0 + l < KMAX ? j0 + l : 0] : 0.0;
      v = warp_sum(v);
      if (lane == l) mine = v;
    }
    scratch[warp * 32 + lane] = mine;
    __syncthreads();
    if (threadIdx.x < 32 && j0 + threadIdx.x < k) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < NWARP; ++w) s += scratch[w * 32 + threadIdx.x];
      out[j0 + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// Last-block detection: returns true in exactly one block per counter after
// all `nblocks` blocks have published their partials.
__device__ __forceinline__ bool last_block(int *counter, int nblocks, int *flag_smem) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    int prev = atomicAdd(counter, 1);
    *flag_smem = (prev == nblocks - 1);
  }
  __syncthreads();
  bool last = *flag_smem != 0;
  if (last) __threadfence();
  return last;
}

// Deterministic reduction by the last block: out[f] = sum_g part[g*stride + f]
// for f < nf, summed in block order g = 0..ng-1 (fixed order, identical on
// every run).  Uses all threads: field f is split over `split` threads whose
// partial sums are then combined in order.
inline __device__ void reduce_fields(const double *part, int ng, int stride, int nf, double *out,
                              double *scratch /* >= NT doubles */) {
  int split = NT / nf;
  if (split < 1) split = 1;
  if (split > 32) split = 32;
  int f = threadIdx.x / split, s = threadIdx.x % split;
  double acc = 0.0;
  if (f < nf) {
    int per = (ng + split - 1) / split;
    int g0 = s * per, g1 = min(ng, g0 + per);
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    int g = g0;
    for (; g + 3 < g1; g += 4) {
      a0 += __ldcg(part + (long long)g * stride + f);
      a1 += __ldcg(part + (long long)(g + 1) * stride + f);
      a2 += __ldcg(part + (long long)(g + 2) * stride + f);
      a3 += __ldcg(part + (long long)(g + 3) * stride + f);
    }
    for (; g < g1; ++g) a0 += __ldcg(part + (long long)g * stride + f);
    acc = (a0 + a1) + (a2 + a3);
  }
  scratch[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < nf && threadIdx.x * 1 < NT) {
    int ff = threadIdx.x;
    if (ff < nf && ff * split < NT) {
      double t = 0.0;
      for (int q = 0; q < split; ++q) t += scratch[ff * split + q];
      out[ff] = t;
    }
  }
  __syncthreads();
}

}  // namespace sdf
