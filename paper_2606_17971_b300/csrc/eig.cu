// eig.cu -- the reference eigensolve on sm_103a: the k smallest eigenpairs
// of A (the operator of the problem, symmetric when there is no convection),
// which are those of S = mass I + wgt A^T A with lambda_S = mass + wgt
// lambda_A^2 (Sec. 2.1.2 Eq. schur), by Chebyshev-filtered subspace iteration
// (Zhou & Saad, 2007: a scaled Chebyshev filter that damps the unwanted
// interval [a, b] of the spectrum, Rayleigh-Ritz on the filtered block).
// The paper computes its reference modes with ARPACK (Sec. 2.2.2) or in
// closed form on tensor-product grids (Sec. 2.2.8); this replaces the former.
//
// The same driver computes the k smallest eigenpairs of the restricted
// operator S_II (App. A.2), applied through the solver's own stencil; the
// file also holds the spectral diagnostics of App. A.1, Sec. 4.1 and App. D
// (active-set distances, operator drift by Lanczos, principal angles) and
// the coarse-grid basis of Sec. 2.2.7.
//
// Every vector operation is FP64 on the GPU; the m x m Rayleigh-Ritz and
// Cholesky factorisations run on the host (m = k + guard <= 320).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <string>
#include <vector>

#include "../../include/sdf.h"
#include "host_linalg.h"
#include "sdf_device.cuh"

// defined in sdf.cu: the operator parameters of a bound problem
const sdf::OpParams *sdf_internal_op(const sdf_problem *p, int *nsm, int *convection);
void sdf_internal_set_error(sdf_problem *p, const char *msg);
const sdf_problem_desc *sdf_internal_desc(const sdf_problem *p, const double **kappa_host);
const void *sdf_internal_modes(const sdf_problem *p, int *k, long long *ld, sdf_dtype *dtype);
sdf_status sdf_internal_apply_S_cols(sdf_problem *p, const double *inst_dev,
                                     const uint8_t *active_dev, const double *u, double *out,
                                     int cols, int mode, cudaStream_t s);

namespace {

using sdf::OpParams;
constexpr int ET = 256;

sdf_status efail(sdf_problem *p, sdf_status s, const char *msg) {
  sdf_internal_set_error(p, msg);
  return s;
}

#define ECK(x)                                                                 \
  do {                                                                         \
    cudaError_t e_ = (x);                                                      \
    if (e_ != cudaSuccess) {                                                   \
      sdf_internal_set_error(p, (std::string(#x) + ": " + cudaGetErrorString(e_)).c_str()); \
      return SDF_ERR_CUDA;                                                     \
    }                                                                          \
  } while (0)

// SplitMix64 (Steele, Lea & Flood, 2014): a counter-based generator; the
// start block entry (g, j) is a uniform value in [-1, 1) from the counter
// seed + (j N + g) * golden
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

__global__ void k_rand_block(double *X, long long N, int m, uint64_t seed) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * m;
       e += (long long)gridDim.x * blockDim.x) {
    const uint64_t r = splitmix64(seed + (uint64_t)e * 0x9e3779b97f4a7c15ULL);
    X[e] = (double)(r >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

// face coefficient of the diffusion operator (constant or from kappa)
__device__ __forceinline__ double fcx(const OpParams &P, int i, int j, int l) {
  return P.fx ? P.fx[i + (long long)(P.nx + 1) * (j + (long long)P.ny * l)] : P.cdiff[0];
}
__device__ __forceinline__ double fcy(const OpParams &P, int i, int j, int l) {
  return P.fy ? P.fy[i + (long long)P.nx * (j + (long long)(P.ny + 1) * l)] : P.cdiff[1];
}
__device__ __forceinline__ double fcz(const OpParams &P, int i, int j, int l) {
  return P.fz ? P.fz[i + (long long)P.nx * (j + (long long)P.ny * l)] : P.cdiff[2];
}

// One step of the three-term recurrence for every column j (blockIdx.y):
// Xn = alpha A Xc + beta Xc + gamma Xp (gamma = 0: Xp is not read).
// A u = sum over the faces of f (u_p - u_nb), u = 0 outside the grid.
__global__ void __launch_bounds__(ET) k_cheb(OpParams P, const double *Xp, const double *Xc,
                                             double *Xn, long long N, double alpha, double beta,
                                             double gamma) {
  const int j = blockIdx.y;
  const double *u = Xc + (long long)j * N;
  for (long long g = blockIdx.x * (long long)ET + threadIdx.x; g < N;
       g += (long long)gridDim.x * ET) {
    const int i = (int)(g % P.nx);
    const long long t = g / P.nx;
    const int jj = (int)(t % P.ny), l = (int)(t / P.ny);
    const double c = u[g];
    double acc = fcx(P, i, jj, l) * (c - (i > 0 ? u[g - 1] : 0.0)) +
                 fcx(P, i + 1, jj, l) * (c - (i + 1 < P.nx ? u[g + 1] : 0.0)) +
                 fcy(P, i, jj, l) * (c - (jj > 0 ? u[g - P.nx] : 0.0)) +
                 fcy(P, i, jj + 1, l) * (c - (jj + 1 < P.ny ? u[g + P.nx] : 0.0));
    if (P.dim == 3) {
      const long long nxy = (long long)P.nx * P.ny;
      acc += fcz(P, i, jj, l) * (c - (l > 0 ? u[g - nxy] : 0.0)) +
             fcz(P, i, jj, l + 1) * (c - (l + 1 < P.nz ? u[g + nxy] : 0.0));
    }
    double v = fma(alpha, acc, beta * c);
    if (gamma != 0.0) v = fma(gamma, Xp[(long long)j * N + g], v);
    Xn[(long long)j * N + g] = v;
  }
}

// Gershgorin bound of A: max over nodes of diag + sum |off-diagonal| = 2 diag
__global__ void k_gershgorin(OpParams P, long long N, double *part) {
  __shared__ double red[ET];
  double mx = 0.0;
  for (long long g = blockIdx.x * (long long)ET + threadIdx.x; g < N;
       g += (long long)gridDim.x * ET) {
    const int i = (int)(g % P.nx);
    const long long t = g / P.nx;
    const int jj = (int)(t % P.ny), l = (int)(t / P.ny);
    double d = fcx(P, i, jj, l) + fcx(P, i + 1, jj, l) + fcy(P, i, jj, l) + fcy(P, i, jj + 1, l);
    if (P.dim == 3) d += fcz(P, i, jj, l) + fcz(P, i, jj, l + 1);
    mx = fmax(mx, 2.0 * d);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = ET / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Gram partials C_c = X^T Y over node chunk c (X, Y column-major N x m):
// 16 x 16 tiles of (i, j), blockIdx.x = chunk
constexpr int GT = 16;
__global__ void __launch_bounds__(256) k_gram2(const double *X, const double *Y, long long N, int m,
                                               int nchunk, double *part) {
  __shared__ double sx[GT][65], sy[GT][65];
  const int ti = blockIdx.y, tj = blockIdx.z;
  const int a = threadIdx.x / GT, c = threadIdx.x % GT;
  const long long per = (N + nchunk - 1) / nchunk;
  const long long g0 = blockIdx.x * per, g1 = min(N, g0 + per);
  double acc = 0.0;
  for (long long gb = g0; gb < g1; gb += 64) {
    for (int e = threadIdx.x; e < GT * 64; e += 256) {
      const int r = e / 64, q = e % 64;
      const long long g = gb + q;
      const int ii = ti * GT + r, jj = tj * GT + r;
      sx[r][q] = (g < g1 && ii < m) ? X[(long long)ii * N + g] : 0.0;
      sy[r][q] = (g < g1 && jj < m) ? Y[(long long)jj * N + g] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < 64; ++q) acc = fma(sx[a][q], sy[c][q], acc);
    __syncthreads();
  }
  const int i = ti * GT + a, j = tj * GT + c;
  if (i < m && j < m) part[((long long)blockIdx.x * m + i) * m + j] = acc;
}

__global__ void k_gram2_reduce(const double *part, int nchunk, int m, double *C) {
  const long long n = (long long)m * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += part[(long long)c * n + e];
    C[e] = s;
  }
}

// Y = X W for a small m x mo matrix W (row-major, in shared memory): per node
// g, Y[j][g] = sum_i X[i][g] W[i][j]
__global__ void __launch_bounds__(128) k_rotate(const double *X, const double *W, long long N, int m,
                                                int mo, double *Y) {
  extern __shared__ double ws[];
  for (int e = threadIdx.x; e < m * mo; e += blockDim.x) ws[e] = W[e];
  __syncthreads();
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= N) return;
  for (int j0 = 0; j0 < mo; j0 += 8) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < m; ++i) {
      const double x = X[(long long)i * N + g];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (j0 + q < mo) acc[q] = fma(x, ws[i * mo + j0 + q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (j0 + q < mo) Y[(long long)(j0 + q) * N + g] = acc[q];
  }
}

// squared norms of AX_j - theta_j X_j for j < k: partials per block
__global__ void k_resid_norms(const double *AX, const double *X, const double *theta, long long N,
                              int k, int nchunk, double *part) {
  __shared__ double red[ET];
  const int j = blockIdx.y;
  const long long per = (N + nchunk - 1) / nchunk;
  const long long g0 = blockIdx.x * per, g1 = min(N, g0 + per);
  const double th = theta[j];
  double s = 0.0;
  for (long long g = g0 + threadIdx.x; g < g1; g += ET) {
    const double r = AX[(long long)j * N + g] - th * X[(long long)j * N + g];
    s = fma(r, r, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int q = ET / 2; q > 0; q >>= 1) {
    if ((int)threadIdx.x < q) red[threadIdx.x] += red[threadIdx.x + q];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long long)j * nchunk + blockIdx.x] = red[0];
}

// Prolongation of r coarse vectors (column-major, Nc rows) to the fine grid:
// each fine node takes the (bi/tri)linear interpolant of the coarse values,
// the coarse node j of a direction sitting at (j + 1) / (nc + 1) and the
// boundary values being zero (Sec. 2.2.7 Eq. prolong).
__global__ void k_prolong(int dim, int nx, int ny, int nz, int cx, int cy, int cz,
                          const double *Xc, int r, double *Xf) {
  const long long N = (long long)nx * ny * nz, Nc = (long long)cx * cy * cz;
  const int j = blockIdx.y;
  for (long long g = blockIdx.x * (long long)ET + threadIdx.x; g < N;
       g += (long long)gridDim.x * ET) {
    const int i = (int)(g % nx);
    const long long t = g / nx;
    const int jj = (int)(t % ny), l = (int)(t / ny);
    int c0[3];
    double w1[3];
    const int fi[3] = {i, jj, l}, fn[3] = {nx, ny, nz}, cn[3] = {cx, cy, cz};
    for (int d = 0; d < 3; ++d) {
      if (d < dim) {
        const double tc = (double)(fi[d] + 1) / (double)(fn[d] + 1) * (double)(cn[d] + 1) - 1.0;
        c0[d] = (int)floor(tc);
        w1[d] = tc - c0[d];
      } else {
        c0[d] = 0;
        w1[d] = 0.0;
      }
    }
    double acc = 0.0;
    for (int corner = 0; corner < (1 << dim); ++corner) {
      double wt = 1.0;
      long long idx = 0, stride = 1;
      bool in = true;
      for (int d = 0; d < dim; ++d) {
        const int a = (corner >> d) & 1;
        const int cidx = c0[d] + a;
        wt *= a ? w1[d] : 1.0 - w1[d];
        in = in && cidx >= 0 && cidx < cn[d];
        idx += (long long)cidx * stride;
        stride *= cn[d];
      }
      if (in && wt != 0.0) acc = fma(wt, Xc[(long long)j * Nc + idx], acc);
    }
    Xf[(long long)j * N + g] = acc;
  }
}

// Block operations on column-major N x m blocks: Gram matrices X^T Y (FP64
// partials per node chunk, summed in chunk order) and rotations X W by a
// small host matrix (in column chunks that fit in shared memory).
struct BlockOps {
  sdf_problem *p;
  cudaStream_t s;
  long long N;
  int nchunk;
  double *part;   // nchunk * m * m doubles
  double *small;  // 2 * m * m doubles
  int mmax;

  sdf_status gram(const double *Xa, const double *Ya, int m, std::vector<double> &C) {
    const int tiles = (m + GT - 1) / GT;
    k_gram2<<<dim3(nchunk, tiles, tiles), 256, 0, s>>>(Xa, Ya, N, m, nchunk, part);
    k_gram2_reduce<<<64, 256, 0, s>>>(part, nchunk, m, small);
    ECK(cudaGetLastError());
    C.resize((size_t)m * m);
    ECK(cudaMemcpyAsync(C.data(), small, sizeof(double) * m * m, cudaMemcpyDeviceToHost, s));
    ECK(cudaStreamSynchronize(s));
    return SDF_OK;
  }
  sdf_status rotate(const double *Xa, const std::vector<double> &W, int m, int mo, double *Yo) {
    const int mc = std::max(8, std::min(mo, (int)((160 * 1024) / (sizeof(double) * m)) / 8 * 8));
    ECK(cudaFuncSetAttribute(k_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * (size_t)m * mc)));
    for (int j0 = 0; j0 < mo; j0 += mc) {
      const int w = std::min(mc, mo - j0);
      std::vector<double> Wc((size_t)m * w);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < w; ++j) Wc[(size_t)i * w + j] = W[(size_t)i * mo + j0 + j];
      double *wd = small + (size_t)mmax * mmax;
      ECK(cudaMemcpyAsync(wd, Wc.data(), sizeof(double) * m * w, cudaMemcpyHostToDevice, s));
      k_rotate<<<(unsigned)((N + 127) / 128), 128, sizeof(double) * (size_t)m * w, s>>>(
          Xa, wd, N, m, w, Yo + (size_t)j0 * N);
      ECK(cudaGetLastError());
      // the host block is reused by the next chunk: wait for this copy
      ECK(cudaStreamSynchronize(s));
    }
    return SDF_OK;
  }
};


size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

int eig_block(int k, const sdf_eig_opts *o) {
  const int guard = o->guard > 0 ? o->guard : std::max(16, k / 2);
  return k + guard;
}

// Xn = a Xn + b Xc + c Xp elementwise over n entries (Xn holds Op Xc on
// entry; Xp is read only when c != 0)
__global__ void k_comb(double *Xn, const double *Xc, const double *Xp, long long n, double a,
                       double b, double c) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double v = fma(a, Xn[e], b * Xc[e]);
    if (c != 0.0) v = fma(c, Xp[e], v);
    Xn[e] = v;
  }
}

// zero the rows on the active set of the m columns of X (column-major N x m)
__global__ void k_mask_rows(double *X, long long N, int m, const uint8_t *mask) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * m;
       e += (long long)gridDim.x * blockDim.x)
    if (mask[e % N]) X[e] = 0.0;
}

// number of inactive nodes (integer atomics: exact and order-independent)
__global__ void k_count_inactive(const uint8_t *mask, long long N, unsigned long long *cnt) {
  unsigned long long c = 0;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N;
       g += (long long)gridDim.x * blockDim.x)
    c += mask[g] == 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// Dot products c_j = V_j . x for the first `cols` columns of V (column-major,
// leading dimension N): partial sums per node chunk, part[j * nchunk + chunk]
__global__ void __launch_bounds__(ET) k_vtw(const double *V, long long N, const double *x,
                                            int nchunk, double *part) {
  __shared__ double red[ET / 32];
  const int j = blockIdx.y;
  const long long per = (N + nchunk - 1) / nchunk;
  const long long g0 = blockIdx.x * per, g1 = min(N, g0 + per);
  const double *v = V + (long long)j * N;
  double s = 0.0;
  for (long long g = g0 + threadIdx.x; g < g1; g += ET) s = fma(v[g], x[g], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < ET / 32; ++q) t += red[q];
    part[(long long)j * nchunk + blockIdx.x] = t;
  }
}

// x -= V c over the first `cols` columns (c in device memory)
__global__ void k_vsub(const double *V, long long N, int cols, const double *c, double *x) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N;
       g += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < cols; ++j) acc = fma(V[(long long)j * N + g], c[j], acc);
    x[g] -= acc;
  }
}

// y = a x + b y (b = 0: y is not read, so it may hold anything)
__global__ void k_axpby(double *y, const double *x, long long N, double a, double b) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N;
       g += (long long)gridDim.x * blockDim.x)
    y[g] = b == 0.0 ? a * x[g] : fma(a, x[g], b * y[g]);
}

// the first k modes (dtype T, leading dimension ld) in FP64 with their rows
// on the active set zeroed: Phi_I in full-grid layout
template <class T> __device__ __forceinline__ double to_f64(T v) { return (double)v; }
template <> __device__ __forceinline__ double to_f64<__nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}
template <class T>
__global__ void k_restrict_modes(const T *phi, long long ld, int k, long long N,
                                 const uint8_t *mask, double *out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * k;
       e += (long long)gridDim.x * blockDim.x) {
    const long long j = e / N, g = e - j * N;
    out[e] = (mask && mask[g]) ? 0.0 : to_f64(phi[j * ld + g]);
  }
}

// Per node chunk (blockIdx.x) and group of DSB instances (blockIdx.y):
// |A_ref sym-diff A_b|, |A_b|, sum_j w_j [A_ref(j) != A_b(j)] and sum_j w_j,
// with w_j = sum_{q<r} phi_q(j)^2 computed once per node for the group (the
// modes are read B / DSB times, the masks once).  The counts are integers
// held in doubles (exact below 2^53).  part[(b nchunk + chunk) 4 + i].
constexpr int DSB = 8;
template <class T>
__global__ void __launch_bounds__(ET) k_diag_sets(const uint8_t *aref, const uint8_t *act, int B,
                                                  long long N, const T *phi, long long ld, int r,
                                                  int nchunk, double *part) {
  constexpr int NV = 3 * DSB + 1;
  __shared__ double red[NV][ET / 32];
  const int b0 = blockIdx.y * DSB;
  const int nb = min(DSB, B - b0);
  const long long per = (N + nchunk - 1) / nchunk;
  const long long g0 = blockIdx.x * per, g1 = min(N, g0 + per);
  double v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.0;
  for (long long g = g0 + threadIdx.x; g < g1; g += ET) {
    const bool x = aref[g] != 0;
    double w = 0.0;
    for (int q = 0; q < r; ++q) {
      const double f = to_f64(phi[(long long)q * ld + g]);
      w = fma(f, f, w);
    }
    v[3 * DSB] += w;
#pragma unroll
    for (int bb = 0; bb < DSB; ++bb) {
      if (bb < nb) {
        const bool y = act[(long long)(b0 + bb) * N + g] != 0;
        v[3 * bb] += (x != y);
        v[3 * bb + 1] += y;
        if (x != y) v[3 * bb + 2] += w;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    if ((threadIdx.x & 31) == 0) red[i][threadIdx.x >> 5] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < 3 * nb) {
    const int bb = threadIdx.x / 3, i = threadIdx.x % 3;
    double t = 0.0, ws = 0.0;
    for (int q = 0; q < ET / 32; ++q) {
      t += red[threadIdx.x][q];
      ws += red[3 * DSB][q];
    }
    double *o = part + ((long long)(b0 + bb) * nchunk + blockIdx.x) * 4;
    o[i] = t;
    if (i == 0) o[3] = ws;
  }
}

// Partial sums over node chunks (blockIdx.x) of ||lam_I||^2 and
// ||lam_I + (S_II y)_I||^2 for one instance: part[2 chunk + {0, 1}]
__global__ void __launch_bounds__(ET) k_relres_parts(const double *lam, const double *sy,
                                                     const uint8_t *act, long long N, int nchunk,
                                                     double *part) {
  __shared__ double red[2][ET / 32];
  const long long per = (N + nchunk - 1) / nchunk;
  const long long g0 = blockIdx.x * per, g1 = min(N, g0 + per);
  double rr = 0.0, bb = 0.0;
  for (long long g = g0 + threadIdx.x; g < g1; g += ET) {
    if (act[g]) continue;
    const double r = lam[g], b = r + sy[g];
    rr = fma(r, r, rr);
    bb = fma(b, b, bb);
  }
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    bb += __shfl_down_sync(0xffffffffu, bb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = rr;
    red[1][threadIdx.x >> 5] = bb;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int q = 0; q < ET / 32; ++q) t += red[threadIdx.x][q];
    part[2 * (long long)blockIdx.x + threadIdx.x] = t;
  }
}

// Orthonormalise the m columns of *A in place: shifted Cholesky-QR, then
// Cholesky-QR twice (Fukaya et al., "shifted CholeskyQR3"); the shift
// 11 (N m + m (m + 1)) u ||A||_F^2 keeps the first factorisation defined
// however ill-conditioned the block is (shift = false: plain CholeskyQR
// three times, which fails on a numerically rank-deficient block).  The
// factor is triangular, so span(Q[:, :r]) = span(A[:, :r]) for every r.
// *tmp is scratch; the two pointers may be swapped.
sdf_status cholqr3(BlockOps &ops, double *&A, double *&tmp, int m, bool shift, const char *what) {
  sdf_problem *p = ops.p;
  for (int rep = 0; rep < 3; ++rep) {
    std::vector<double> G, L, Wt;
    sdf_status e = ops.gram(A, A, m, G);
    if (e != SDF_OK) return e;
    if (rep == 0 && shift) {
      double tr = 0.0;
      for (int i = 0; i < m; ++i) tr += G[(size_t)i * m + i];
      const double sh = 11.0 * ((double)ops.N * m + (double)m * (m + 1)) * 1.1102230246251565e-16 * tr;
      for (int i = 0; i < m; ++i) G[(size_t)i * m + i] += sh;
    }
    if (!hla::cholesky(m, G, L)) return efail(p, SDF_ERR_NOT_SPD, what);
    hla::inv_lower_transpose(m, L, Wt);
    e = ops.rotate(A, Wt, m, m, tmp);
    if (e != SDF_OK) return e;
    std::swap(A, tmp);
  }
  return SDF_OK;
}

// Xn = a Op(Xc) + b Xc + c Xp on `cols` columns (c = 0: Xp is not read)
using ApplyFn = std::function<sdf_status(const double *Xp, const double *Xc, double *Xn, int cols,
                                         double a, double b, double c)>;

struct ChebResult {
  std::vector<double> theta;  // Ritz values of the block, ascending
  int iters = 0, converged = 0;
  double maxrel = INFINITY;
  int64_t matvecs = 0;
};

// Chebyshev-filtered subspace iteration (Zhou & Saad) for the k smallest
// eigenpairs of a symmetric positive semi-definite operator whose spectrum
// lies in [0, bmax]: block of m = k + guard columns, adaptive filter degree,
// shifted CholeskyQR3, Rayleigh-Ritz on the host.  With `mask`, the start
// block is zero on the masked rows and the operator keeps it so.  The k
// wanted vectors are copied to phi_dev (leading dimension ld).
sdf_status cheb_eigs(sdf_problem *p, cudaStream_t s, long long N, int nsm, int k,
                     const sdf_eig_opts *o, const ApplyFn &op, double bmax, const uint8_t *mask,
                     void *ws, double *phi_dev, int64_t ld, ChebResult &res) {
  const int m = eig_block(k, o);
  const int nchunk = 2 * nsm;
  char *w = (char *)ws;
  size_t off = 0;
  auto take = [&](size_t b) {
    char *at = w + off;
    off += al256(b);
    return at;
  };
  double *X = (double *)take(sizeof(double) * (size_t)N * m);
  double *Y = (double *)take(sizeof(double) * (size_t)N * m);
  double *Z = (double *)take(sizeof(double) * (size_t)N * m);
  double *AX = (double *)take(sizeof(double) * (size_t)N * m);
  double *part = (double *)take(sizeof(double) * (size_t)nchunk * m * m);
  double *small = (double *)take(sizeof(double) * (size_t)m * m * 2);
  double *theta_d = (double *)take(sizeof(double) * (size_t)m);
  auto apply = [&](const double *Xp, const double *Xc, double *Xn, int cols, double a, double b,
                   double c) -> sdf_status {
    res.matvecs += cols;
    return op(Xp, Xc, Xn, cols, a, b, c);
  };
  BlockOps ops{p, s, N, nchunk, part, small, m};
  std::vector<double> &theta = res.theta;
  theta.assign(m, 0.0);
  std::vector<double> V, H;
  // Rayleigh-Ritz on the orthonormal block *Xb: *Xb <- Xb V, AX = Op Xb,
  // theta ascending
  auto rayleigh_ritz = [&](double *&Xb, double *&tmp) -> sdf_status {
    sdf_status e = apply(nullptr, Xb, AX, m, 1.0, 0.0, 0.0);
    if (e != SDF_OK) return e;
    e = ops.gram(Xb, AX, m, H);
    if (e != SDF_OK) return e;
    for (int i = 0; i < m; ++i)  // symmetrise the rounding
      for (int j = i + 1; j < m; ++j) {
        const double a = 0.5 * (H[(size_t)i * m + j] + H[(size_t)j * m + i]);
        H[(size_t)i * m + j] = H[(size_t)j * m + i] = a;
      }
    std::vector<double> wv, Vd;
    hla::jacobi_eig(m, H, wv, Vd);  // descending
    V.assign((size_t)m * m, 0.0);
    for (int j = 0; j < m; ++j) {
      theta[j] = wv[m - 1 - j];
      for (int i = 0; i < m; ++i) V[(size_t)i * m + j] = Vd[(size_t)i * m + (m - 1 - j)];
    }
    e = ops.rotate(Xb, V, m, m, tmp);
    if (e != SDF_OK) return e;
    std::swap(Xb, tmp);
    e = ops.rotate(AX, V, m, m, tmp);  // Op (Xb V) = (Op Xb) V
    if (e != SDF_OK) return e;
    ECK(cudaMemcpyAsync(AX, tmp, sizeof(double) * (size_t)N * m, cudaMemcpyDeviceToDevice, s));
    return SDF_OK;
  };

  // start block
  k_rand_block<<<nsm * 8, ET, 0, s>>>(X, N, m, o->seed);
  if (mask) k_mask_rows<<<nsm * 8, ET, 0, s>>>(X, N, m, mask);
  ECK(cudaGetLastError());
  double *Xb = X, *T1 = Y, *T2 = Z;
  sdf_status e = cholqr3(ops, Xb, T1, m, true, "eig: block lost rank");
  if (e != SDF_OK) return e;
  e = rayleigh_ritz(Xb, T1);
  if (e != SDF_OK) return e;
  int it = 0;
  std::vector<double> rn(k);
  for (it = 1; it <= o->max_iter; ++it) {
    // scaled Chebyshev filter on [a, bmax], scaled at a0 (Zhou & Saad)
    const double a = std::min(theta[m - 1], 0.5 * bmax), a0 = theta[0];
    const double ee = 0.5 * (bmax - a), cc = 0.5 * (bmax + a);
    // degree of this pass: the filter grows the component at a0 by
    // rho = |x| + sqrt(x^2 - 1), x = (a0 - c) / e, per degree relative to the
    // block's top Ritz value; at most 1e6 over the pass, so that the filtered
    // block stays numerically of full rank
    const double x0 = std::fabs((a0 - cc) / ee);
    const double rho = x0 + std::sqrt(std::max(0.0, x0 * x0 - 1.0));
    const int deg = rho > 1.0 ? std::max(2, std::min(o->degree, (int)(std::log(1e6) / std::log(rho))))
                              : o->degree;
    double sigma = ee / (a0 - cc);
    const double tau = 2.0 / sigma;
    // T1 = (sigma / e) (Op Xb - c Xb)
    e = apply(nullptr, Xb, T1, m, sigma / ee, -cc * sigma / ee, 0.0);
    if (e != SDF_OK) return e;
    double *prev = Xb, *cur = T1, *nxt = T2;
    for (int d = 2; d <= deg; ++d) {
      const double sn = 1.0 / (tau - sigma);
      e = apply(prev, cur, nxt, m, 2.0 * sn / ee, -2.0 * sn * cc / ee, -sigma * sn);
      if (e != SDF_OK) return e;
      sigma = sn;
      double *t = prev;
      prev = cur;
      cur = nxt;
      nxt = t;
    }
    // the filtered block is `cur`; the other two buffers are scratch
    Xb = cur;
    T1 = prev;
    T2 = nxt;
    e = cholqr3(ops, Xb, T1, m, true, "eig: block lost rank");
    if (e != SDF_OK) return e;
    e = rayleigh_ritz(Xb, T1);
    if (e != SDF_OK) return e;
    // residuals of the k wanted pairs
    ECK(cudaMemcpyAsync(theta_d, theta.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    k_resid_norms<<<dim3(nchunk, k), ET, 0, s>>>(AX, Xb, theta_d, N, k, nchunk, part);
    ECK(cudaGetLastError());
    std::vector<double> rp((size_t)k * nchunk);
    ECK(cudaMemcpyAsync(rp.data(), part, sizeof(double) * k * nchunk, cudaMemcpyDeviceToHost, s));
    ECK(cudaStreamSynchronize(s));
    res.maxrel = 0.0;
    for (int j = 0; j < k; ++j) {
      double r2 = 0.0;
      for (int c = 0; c < nchunk; ++c) r2 += rp[(size_t)j * nchunk + c];
      rn[j] = std::sqrt(r2);
      res.maxrel = std::max(res.maxrel, rn[j] / std::fabs(theta[j]));
    }
    if (res.maxrel <= o->tol) {
      res.converged = 1;
      break;
    }
  }
  res.iters = std::min(it, o->max_iter);
  // output: the k wanted vectors (unit norm, column-major with leading dim ld)
  ECK(cudaMemcpy2DAsync(phi_dev, sizeof(double) * ld, Xb, sizeof(double) * N, sizeof(double) * N, k,
                        cudaMemcpyDeviceToDevice, s));
  ECK(cudaStreamSynchronize(s));
  return SDF_OK;
}

// Number of eigenvalues below x of the symmetric tridiagonal T (diagonal al,
// off-diagonal be), by the signs of the pivots of T - x I (Sturm sequence;
// Golub & Van Loan, Sec. 8.4); a zero pivot is replaced by a tiny one.
int sturm_count(const std::vector<double> &al, const std::vector<double> &be, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t i = 0; i < al.size(); ++i) {
    const double b2 = i > 0 ? be[i - 1] * be[i - 1] : 0.0;
    q = (al[i] - x) - (i > 0 ? b2 / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// The smallest and largest eigenvalues of T by bisection on the Sturm count
// inside the Gershgorin interval (to the spacing of doubles).
void tridiag_extremes(const std::vector<double> &al, const std::vector<double> &be, double &lo_out,
                      double &hi_out) {
  const size_t m = al.size();
  double lo = INFINITY, hi = -INFINITY;
  for (size_t i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(be[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(be[i]) : 0.0);
    lo = std::min(lo, al[i] - r);
    hi = std::max(hi, al[i] + r);
  }
  auto bisect = [&](int target) {  // the smallest x with count(x) > target
    double a = lo, b = hi;
    for (int it = 0; it < 200 && b - a > 0.0; ++it) {
      const double c = 0.5 * (a + b);
      if (c <= a || c >= b) break;
      if (sturm_count(al, be, c) > target) b = c;
      else a = c;
    }
    return 0.5 * (a + b);
  };
  lo_out = bisect(0);
  hi_out = bisect((int)m - 1);
}

// Largest |eigenvalue| of a symmetric operator on N-vectors by Lanczos with
// full reorthogonalisation (classical Gram-Schmidt applied twice per step),
// from the SplitMix64 start vector `seed`.  Stops after `steps` steps, at N,
// or when the new residual norm beta falls to 1e-14 of the largest
// coefficient seen (an invariant subspace).  V holds steps + 1 columns of N;
// x is one N-vector of scratch; cdev at least steps + 1 doubles.
sdf_status lanczos_absmax(sdf_problem *p, cudaStream_t s, long long N, int nsm, int steps,
                          uint64_t seed, const std::function<sdf_status(const double *, double *)> &op,
                          double *V, double *x, double *part, double *cdev, double &out) {
  const int nchunk = 2 * nsm;
  const unsigned grid = (unsigned)std::min<long long>((N + ET - 1) / ET, nsm * 8LL);
  auto dots = [&](const double *Vb, int cols, const double *y, std::vector<double> &c) -> sdf_status {
    k_vtw<<<dim3(nchunk, cols), ET, 0, s>>>(Vb, N, y, nchunk, part);
    ECK(cudaGetLastError());
    std::vector<double> pp((size_t)cols * nchunk);
    ECK(cudaMemcpyAsync(pp.data(), part, sizeof(double) * pp.size(), cudaMemcpyDeviceToHost, s));
    ECK(cudaStreamSynchronize(s));
    c.assign(cols, 0.0);
    for (int j = 0; j < cols; ++j)
      for (int q = 0; q < nchunk; ++q) c[j] += pp[(size_t)j * nchunk + q];
    return SDF_OK;
  };
  k_rand_block<<<grid, ET, 0, s>>>(V, N, 1, seed);
  ECK(cudaGetLastError());
  std::vector<double> c, c2;
  sdf_status e = dots(V, 1, V, c);
  if (e != SDF_OK) return e;
  k_axpby<<<grid, ET, 0, s>>>(V, V, N, 1.0 / std::sqrt(c[0]), 0.0);
  std::vector<double> al, be;
  double scale = 0.0;
  const int jmax = (int)std::min<long long>(steps, N);
  for (int j = 0; j < jmax; ++j) {
    double *vj = V + (size_t)j * N;
    e = op(vj, x);
    if (e != SDF_OK) return e;
    double alpha = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      e = dots(V, j + 1, x, c);
      if (e != SDF_OK) return e;
      alpha += c[j];
      ECK(cudaMemcpyAsync(cdev, c.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, s));
      k_vsub<<<grid, ET, 0, s>>>(V, N, j + 1, cdev, x);
      ECK(cudaGetLastError());
    }
    e = dots(x, 1, x, c2);
    if (e != SDF_OK) return e;
    const double beta = std::sqrt(c2[0]);
    al.push_back(alpha);
    scale = std::max(scale, std::max(std::fabs(alpha), beta));
    if (j + 1 == jmax || beta <= 1e-14 * scale) break;
    be.push_back(beta);
    k_axpby<<<grid, ET, 0, s>>>(V + (size_t)(j + 1) * N, x, N, 1.0 / beta, 0.0);
    ECK(cudaGetLastError());
  }
  double lo = 0.0, hi = 0.0;
  tridiag_extremes(al, be, lo, hi);
  out = std::max(std::fabs(lo), std::fabs(hi));
  return SDF_OK;
}

}  // namespace

extern "C" {

void sdf_default_eig_opts(sdf_eig_opts *o) {
  if (!o) return;
  o->tol = 1e-6;
  o->degree = 60;
  o->guard = 0;
  o->max_iter = 400;
  o->seed = 20260;
}

sdf_status sdf_eig_workspace_size(const sdf_problem *p, int k, const sdf_eig_opts *o,
                                  size_t *bytes) {
  if (!p || !o || !bytes || k < 1 || k > SDF_MAX_K) return SDF_ERR_INVALID_ARG;
  int nsm = 148, conv = 0;
  const OpParams *P = sdf_internal_op(p, &nsm, &conv);
  if (!P) return SDF_ERR_INVALID_ARG;
  const int m = eig_block(k, o);
  if (m > 320) return SDF_ERR_INVALID_ARG;
  const long long N = P->N;
  const int nchunk = 2 * nsm;
  size_t b = 4 * al256(sizeof(double) * (size_t)N * m);
  b += al256(sizeof(double) * (size_t)nchunk * m * m);
  b += al256(sizeof(double) * (size_t)m * m * 2);
  b += al256(sizeof(double) * (size_t)m);
  *bytes = b;
  return SDF_OK;
}

static void fill_eig_stats(sdf_eig_stats *stats, const ChebResult &r,
                           std::chrono::steady_clock::time_point t0) {
  if (!stats) return;
  stats->iters = r.iters;
  stats->converged = r.converged;
  stats->max_rel_resid = r.maxrel;
  stats->matvecs = r.matvecs;
  stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

sdf_status sdf_reference_modes_eig(sdf_problem *p, int k, const sdf_eig_opts *o, double *phi_dev,
                                   int64_t ld, double *lambda_S_host, double *lambda_A_host,
                                   sdf_eig_stats *stats, void *ws, size_t ws_bytes, void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  sdf_eig_opts def;
  sdf_default_eig_opts(&def);
  if (!o) o = &def;
  size_t need = 0;
  if (sdf_eig_workspace_size(p, k, o, &need) != SDF_OK)
    return efail(p, SDF_ERR_INVALID_ARG, "eig: bad k, options or problem (k + guard <= 320)");
  int nsm = 148, conv = 0;
  const OpParams P = *sdf_internal_op(p, &nsm, &conv);
  if (conv) return efail(p, SDF_ERR_UNSUPPORTED, "eig: A with convection is not symmetric");
  if (P.csr_rp) return efail(p, SDF_ERR_UNSUPPORTED, "eig: the filter runs on the grid's A");
  if (!phi_dev || ld < P.N || !ws || ((uintptr_t)ws & 255) != 0)
    return efail(p, SDF_ERR_INVALID_ARG, "eig: bad output or workspace pointer");
  if (ws_bytes < need) return efail(p, SDF_ERR_WORKSPACE, "eig: workspace too small");
  if (o->degree < 2 || o->max_iter < 1 || !(o->tol > 0))
    return efail(p, SDF_ERR_INVALID_ARG, "eig: bad options");
  const auto t_start = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = P.N;
  const int nchunk = 2 * nsm;
  // spectrum bound of A (Gershgorin), into the partials area of the workspace
  double *gpart = (double *)((char *)ws + 4 * al256(sizeof(double) * (size_t)N * eig_block(k, o)));
  k_gershgorin<<<nchunk, ET, 0, s>>>(P, N, gpart);
  ECK(cudaGetLastError());
  std::vector<double> gp(nchunk);
  ECK(cudaMemcpyAsync(gp.data(), gpart, sizeof(double) * nchunk, cudaMemcpyDeviceToHost, s));
  ECK(cudaStreamSynchronize(s));
  const double bmax = 1.01 * *std::max_element(gp.begin(), gp.end());
  // the operator: A by its stencil (the eigenvectors of S are those of A)
  ApplyFn opA = [&](const double *Xp, const double *Xc, double *Xn, int cols, double a, double b,
                    double c) -> sdf_status {
    const dim3 g((unsigned)std::min<long long>((N + ET - 1) / ET, nsm * 4LL), cols);
    k_cheb<<<g, ET, 0, s>>>(P, Xp, Xc, Xn, N, a, b, c);
    ECK(cudaGetLastError());
    return SDF_OK;
  };
  ChebResult r;
  sdf_status e = cheb_eigs(p, s, N, nsm, k, o, opA, bmax, nullptr, ws, phi_dev, ld, r);
  if (e != SDF_OK) return e;
  for (int j = 0; j < k; ++j) {
    if (lambda_A_host) lambda_A_host[j] = r.theta[j];
    if (lambda_S_host) lambda_S_host[j] = P.mass + P.wgt * r.theta[j] * r.theta[j];
  }
  fill_eig_stats(stats, r, t_start);
  return r.converged ? SDF_OK : efail(p, SDF_ERR_CG_MAXIT, "eig: not converged within max_iter");
}

void sdf_default_restricted_eig_opts(int k, sdf_eig_opts *o) {
  if (!o) return;
  sdf_default_eig_opts(o);
  // S_II's low spectrum is that of A squared and compressed against a bound
  // of wgt ||A||^2, so each filter degree gains about the square root of
  // what it gains on A: a longer filter and a wider guard
  o->degree = 200;
  o->guard = std::max(32, k / 2);
  o->tol = 1e-8;
}

sdf_status sdf_restricted_eig_workspace_size(const sdf_problem *p, int k, const sdf_eig_opts *o,
                                             size_t *bytes) {
  sdf_eig_opts def;
  sdf_default_restricted_eig_opts(k, &def);
  if (!o) o = &def;
  size_t b = 0;
  const sdf_status e = sdf_eig_workspace_size(p, k, o, &b);
  if (e != SDF_OK) return e;
  *bytes = b + al256(sizeof(unsigned long long));
  return SDF_OK;
}

sdf_status sdf_restricted_modes_eig(sdf_problem *p, const double *inst_dev,
                                    const uint8_t *active_dev, int k, const sdf_eig_opts *o,
                                    double *phi_dev, int64_t ld, double *lambda_host,
                                    sdf_eig_stats *stats, void *ws, size_t ws_bytes,
                                    void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  sdf_eig_opts def;
  sdf_default_restricted_eig_opts(k, &def);
  if (!o) o = &def;
  size_t need = 0;
  if (sdf_restricted_eig_workspace_size(p, k, o, &need) != SDF_OK)
    return efail(p, SDF_ERR_INVALID_ARG, "restricted eig: bad k, options or problem");
  int nsm = 148, conv = 0;
  const OpParams P = *sdf_internal_op(p, &nsm, &conv);
  if (!inst_dev || !active_dev || !phi_dev || ld < P.N || !ws || ((uintptr_t)ws & 255) != 0)
    return efail(p, SDF_ERR_INVALID_ARG, "restricted eig: bad pointer");
  if (P.csr_rp)
    return efail(p, SDF_ERR_UNSUPPORTED, "restricted eig: the spectrum bound uses the grid's A");
  if (ws_bytes < need) return efail(p, SDF_ERR_WORKSPACE, "restricted eig: workspace too small");
  if (o->degree < 2 || o->max_iter < 1 || !(o->tol > 0))
    return efail(p, SDF_ERR_INVALID_ARG, "restricted eig: bad options");
  const auto t_start = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = P.N;
  const int m = eig_block(k, o);
  const int nchunk = 2 * nsm;
  size_t eb = 0;
  sdf_eig_workspace_size(p, k, o, &eb);
  unsigned long long *cnt = (unsigned long long *)((char *)ws + eb);
  // |I| >= m, or the block cannot stay of full rank on I
  ECK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  k_count_inactive<<<nsm * 4, ET, 0, s>>>(active_dev, N, cnt);
  ECK(cudaGetLastError());
  unsigned long long nI = 0;
  ECK(cudaMemcpyAsync(&nI, cnt, sizeof(nI), cudaMemcpyDeviceToHost, s));
  // spectrum bound: ||A||_2 <= max row sum of |A| (and column sum, the same
  // bound here): twice the diffusion face sum (Gershgorin kernel) plus
  // 2 sum_d |b_d| / h_d for the upwind convection of this instance, and
  // 2 / dt along the time axis of a space-time problem
  double *gpart = (double *)((char *)ws + 4 * al256(sizeof(double) * (size_t)N * m));
  k_gershgorin<<<nchunk, ET, 0, s>>>(P, N, gpart);
  ECK(cudaGetLastError());
  std::vector<double> gp(nchunk);
  double inst_h[SDF_INSTANCE_DOUBLES];
  ECK(cudaMemcpyAsync(gp.data(), gpart, sizeof(double) * nchunk, cudaMemcpyDeviceToHost, s));
  ECK(cudaMemcpyAsync(inst_h, inst_dev, sizeof(inst_h), cudaMemcpyDeviceToHost, s));
  ECK(cudaStreamSynchronize(s));
  if ((long long)nI < m)
    return efail(p, SDF_ERR_INVALID_ARG, "restricted eig: fewer inactive nodes than k + guard");
  double bA = *std::max_element(gp.begin(), gp.end());
  for (int d = 0; d < P.dim; ++d) {
    if (P.time_axis && d == 2) bA += 2.0 * P.cb_t;  // the implicit Euler difference
    else if (P.inst_conv) bA += 2.0 * std::fabs(inst_h[4 + d]) * P.inv_h[d];
  }
  const double bmax = 1.01 * (P.mass + P.wgt * bA * bA);
  // the operator: S_II through the solver's own stencil (mode 0) on the
  // whole block in one launch, then the three-term combination
  ApplyFn opS = [&](const double *Xp, const double *Xc, double *Xn, int cols, double a, double b,
                    double c) -> sdf_status {
    const sdf_status e = sdf_internal_apply_S_cols(p, inst_dev, active_dev, Xc, Xn, cols, 0, s);
    if (e != SDF_OK) return e;
    if (a != 1.0 || b != 0.0 || c != 0.0) {
      k_comb<<<nsm * 8, ET, 0, s>>>(Xn, Xc, Xp, N * cols, a, b, c);
      ECK(cudaGetLastError());
    }
    return SDF_OK;
  };
  ChebResult r;
  sdf_status e = cheb_eigs(p, s, N, nsm, k, o, opS, bmax, active_dev, ws, phi_dev, ld, r);
  if (e != SDF_OK) return e;
  if (lambda_host)
    for (int j = 0; j < k; ++j) lambda_host[j] = r.theta[j];
  fill_eig_stats(stats, r, t_start);
  return r.converged ? SDF_OK
                     : efail(p, SDF_ERR_CG_MAXIT, "restricted eig: not converged within max_iter");
}

static int diag_chunks(long long N, int nsm) {
  return (int)std::max<long long>(1, std::min<long long>((N + 4LL * ET - 1) / (4LL * ET), 2LL * nsm));
}

sdf_status sdf_diag_sets_workspace_size(const sdf_problem *p, int B, size_t *bytes) {
  int nsm = 148, conv = 0;
  const OpParams *P = p ? sdf_internal_op(p, &nsm, &conv) : nullptr;
  if (!P || !bytes || B < 1) return SDF_ERR_INVALID_ARG;
  *bytes = al256(sizeof(double) * 4 * (size_t)B * diag_chunks(P->N, nsm));
  return SDF_OK;
}

sdf_status sdf_diag_active_sets(sdf_problem *p, const uint8_t *active_ref_dev,
                                const uint8_t *active_dev, int B, int r, int64_t *sym_diff_host,
                                int64_t *n_active_host, double *delta_host, double *rho_host,
                                double *delta_w_host, void *ws, size_t ws_bytes, void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  size_t need = 0;
  if (sdf_diag_sets_workspace_size(p, B, &need) != SDF_OK)
    return efail(p, SDF_ERR_INVALID_ARG, "diag sets: unbound problem or B < 1");
  int nsm = 148, conv = 0;
  const OpParams P = *sdf_internal_op(p, &nsm, &conv);
  if (!active_ref_dev || !active_dev || !ws || ((uintptr_t)ws & 255) != 0)
    return efail(p, SDF_ERR_INVALID_ARG, "diag sets: bad pointer");
  if (ws_bytes < need) return efail(p, SDF_ERR_WORKSPACE, "diag sets: workspace too small");
  int k = 0;
  long long ld = 0;
  sdf_dtype dt = SDF_F64;
  const void *phi = sdf_internal_modes(p, &k, &ld, &dt);
  if (r < 0 || (r > 0 && (!phi || r > k)))
    return efail(p, SDF_ERR_INVALID_ARG, "diag sets: r must be 0 or at most the registered modes");
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = P.N;
  const int nchunk = diag_chunks(N, nsm);
  double *part = (double *)ws;
  const dim3 g(nchunk, (B + DSB - 1) / DSB);
  if (r == 0 || dt == SDF_F64)
    k_diag_sets<double><<<g, ET, 0, s>>>(active_ref_dev, active_dev, B, N, (const double *)phi, ld,
                                         r, nchunk, part);
  else if (dt == SDF_F32)
    k_diag_sets<float><<<g, ET, 0, s>>>(active_ref_dev, active_dev, B, N, (const float *)phi, ld,
                                        r, nchunk, part);
  else
    k_diag_sets<__nv_bfloat16><<<g, ET, 0, s>>>(active_ref_dev, active_dev, B, N,
                                                (const __nv_bfloat16 *)phi, ld, r, nchunk, part);
  ECK(cudaGetLastError());
  std::vector<double> pp((size_t)4 * B * nchunk);
  ECK(cudaMemcpyAsync(pp.data(), part, sizeof(double) * pp.size(), cudaMemcpyDeviceToHost, s));
  ECK(cudaStreamSynchronize(s));
  for (int b = 0; b < B; ++b) {
    double t[4] = {0, 0, 0, 0};
    for (int c = 0; c < nchunk; ++c)
      for (int i = 0; i < 4; ++i) t[i] += pp[((size_t)b * nchunk + c) * 4 + i];
    if (sym_diff_host) sym_diff_host[b] = (int64_t)t[0];
    if (n_active_host) n_active_host[b] = (int64_t)t[1];
    if (delta_host) delta_host[b] = t[0] / (double)N;
    if (rho_host) rho_host[b] = t[1] / (double)N;
    if (delta_w_host && r > 0) delta_w_host[b] = t[3] > 0.0 ? t[2] / t[3] : 0.0;
  }
  return SDF_OK;
}

sdf_status sdf_diag_drift_workspace_size(const sdf_problem *p, int steps, size_t *bytes) {
  int nsm = 148, conv = 0;
  const OpParams *P = p ? sdf_internal_op(p, &nsm, &conv) : nullptr;
  if (!P || !bytes || steps < 1 || steps > 1024) return SDF_ERR_INVALID_ARG;
  const long long N = P->N;
  *bytes = al256(sizeof(double) * (size_t)N * (steps + 1)) + 3 * al256(sizeof(double) * (size_t)N) +
           al256(sizeof(double) * (size_t)2 * nsm * (steps + 1)) +
           al256(sizeof(double) * (size_t)(steps + 1));
  return SDF_OK;
}

sdf_status sdf_diag_drift(sdf_problem *p, const double *inst_ref_dev, const double *inst_dev,
                          int B, int steps, double *eps_host, double *norm_ref_host, void *ws,
                          size_t ws_bytes, void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  size_t need = 0;
  if (sdf_diag_drift_workspace_size(p, steps, &need) != SDF_OK)
    return efail(p, SDF_ERR_INVALID_ARG, "diag drift: unbound problem or steps not in [1, 1024]");
  int nsm = 148, conv = 0;
  const OpParams P = *sdf_internal_op(p, &nsm, &conv);
  if (!inst_ref_dev || (B > 0 && (!inst_dev || !eps_host)) || B < 0 || !ws ||
      ((uintptr_t)ws & 255) != 0)
    return efail(p, SDF_ERR_INVALID_ARG, "diag drift: bad pointer or B");
  if (ws_bytes < need) return efail(p, SDF_ERR_WORKSPACE, "diag drift: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = P.N;
  char *w = (char *)ws;
  double *V = (double *)w;
  w += al256(sizeof(double) * (size_t)N * (steps + 1));
  double *x = (double *)w;
  w += al256(sizeof(double) * (size_t)N);
  double *t1 = (double *)w;
  w += al256(sizeof(double) * (size_t)N);
  double *t2 = (double *)w;
  w += al256(sizeof(double) * (size_t)N);
  double *part = (double *)w;
  w += al256(sizeof(double) * (size_t)2 * nsm * (steps + 1));
  double *cdev = (double *)w;
  const unsigned grid = (unsigned)std::min<long long>((N + ET - 1) / ET, nsm * 8LL);
  const uint64_t seed = 0x5dee7ULL;
  // ||S(ref)||_2: S(ref) is positive definite, its largest eigenvalue
  double nref = 0.0;
  sdf_status e = lanczos_absmax(
      p, s, N, nsm, steps, seed,
      [&](const double *v, double *y) {
        return sdf_apply_S(p, inst_ref_dev, nullptr, v, y, 1, nullptr, 0, stream);
      },
      V, x, part, cdev, nref);
  if (e != SDF_OK) return e;
  if (norm_ref_host) *norm_ref_host = nref;
  for (int b = 0; b < B; ++b) {
    const double *ib = inst_dev + (size_t)b * SDF_INSTANCE_DOUBLES;
    double nd = 0.0;
    e = lanczos_absmax(
        p, s, N, nsm, steps, seed,
        [&](const double *v, double *y) -> sdf_status {
          sdf_status q = sdf_apply_S(p, inst_ref_dev, nullptr, v, t1, 1, nullptr, 0, stream);
          if (q != SDF_OK) return q;
          q = sdf_apply_S(p, ib, nullptr, v, t2, 1, nullptr, 0, stream);
          if (q != SDF_OK) return q;
          ECK(cudaMemcpyAsync(y, t1, sizeof(double) * (size_t)N, cudaMemcpyDeviceToDevice, s));
          k_axpby<<<grid, ET, 0, s>>>(y, t2, N, -1.0, 1.0);
          ECK(cudaGetLastError());
          return SDF_OK;
        },
        V, x, part, cdev, nd);
    if (e != SDF_OK) return e;
    eps_host[b] = nref > 0.0 ? nd / nref : 0.0;
  }
  return SDF_OK;
}

sdf_status sdf_diag_relres_workspace_size(const sdf_problem *p, size_t *bytes) {
  int nsm = 148, conv = 0;
  const OpParams *P = p ? sdf_internal_op(p, &nsm, &conv) : nullptr;
  if (!P || !bytes) return SDF_ERR_INVALID_ARG;
  *bytes = al256(sizeof(double) * (size_t)P->N) + al256(sizeof(double) * 2 * (size_t)2 * nsm);
  return SDF_OK;
}

sdf_status sdf_diag_relres(sdf_problem *p, const double *inst_dev, int B, const double *y_dev,
                           const double *lambda_dev, const uint8_t *active_dev,
                           double *relres_host, void *ws, size_t ws_bytes, void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  size_t need = 0;
  if (sdf_diag_relres_workspace_size(p, &need) != SDF_OK)
    return efail(p, SDF_ERR_INVALID_ARG, "diag relres: unbound problem");
  int nsm = 148, conv = 0;
  const OpParams P = *sdf_internal_op(p, &nsm, &conv);
  if (B < 1 || !y_dev || !lambda_dev || !active_dev || !relres_host || !ws ||
      ((uintptr_t)ws & 255) != 0 || (!inst_dev && P.inst_conv))
    return efail(p, SDF_ERR_INVALID_ARG, "diag relres: bad pointer or B");
  if (ws_bytes < need) return efail(p, SDF_ERR_WORKSPACE, "diag relres: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = P.N;
  const int nchunk = 2 * nsm;
  double *sy = (double *)ws;
  double *part = (double *)((char *)ws + al256(sizeof(double) * (size_t)N));
  std::vector<double> pp(2 * (size_t)nchunk);
  for (int b = 0; b < B; ++b) {
    // the instance row is read only for its convection velocity; without
    // per-instance convection any valid pointer stands in for it
    const double *ib = inst_dev ? inst_dev + (size_t)b * SDF_INSTANCE_DOUBLES : y_dev;
    const uint8_t *ab = active_dev + (size_t)b * N;
    // S_II y_I (mode 0 reads y as zero on A and writes zero there)
    sdf_status e = sdf_internal_apply_S_cols(p, ib, ab, y_dev + (size_t)b * N, sy, 1, 0, s);
    if (e != SDF_OK) return e;
    k_relres_parts<<<nchunk, ET, 0, s>>>(lambda_dev + (size_t)b * N, sy, ab, N, nchunk, part);
    ECK(cudaGetLastError());
    ECK(cudaMemcpyAsync(pp.data(), part, sizeof(double) * pp.size(), cudaMemcpyDeviceToHost, s));
    ECK(cudaStreamSynchronize(s));
    double rr = 0.0, bb = 0.0;
    for (int c = 0; c < nchunk; ++c) {
      rr += pp[2 * (size_t)c];
      bb += pp[2 * (size_t)c + 1];
    }
    relres_host[b] = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
  }
  return SDF_OK;
}

sdf_status sdf_diag_angles_workspace_size(const sdf_problem *p, int k, size_t *bytes) {
  int nsm = 148, conv = 0;
  const OpParams *P = p ? sdf_internal_op(p, &nsm, &conv) : nullptr;
  if (!P || !bytes || k < 1 || k > SDF_MAX_K) return SDF_ERR_INVALID_ARG;
  const long long N = P->N;
  *bytes = 3 * al256(sizeof(double) * (size_t)N * k) +
           al256(sizeof(double) * (size_t)2 * nsm * k * k) + al256(sizeof(double) * (size_t)2 * k * k);
  return SDF_OK;
}

sdf_status sdf_diag_angles(sdf_problem *p, const uint8_t *active_dev, const double *V_dev,
                           int64_t ldv, int k, double *theta_host, double *sorted_host, void *ws,
                           size_t ws_bytes, void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  size_t need = 0;
  if (sdf_diag_angles_workspace_size(p, k, &need) != SDF_OK)
    return efail(p, SDF_ERR_INVALID_ARG, "diag angles: unbound problem or bad k");
  int nsm = 148, conv = 0;
  const OpParams P = *sdf_internal_op(p, &nsm, &conv);
  int kr = 0;
  long long ld = 0;
  sdf_dtype dt = SDF_F64;
  const void *phi = sdf_internal_modes(p, &kr, &ld, &dt);
  if (!phi || k > kr) return efail(p, SDF_ERR_INVALID_ARG, "diag angles: k above the registered modes");
  if (!active_dev || !V_dev || ldv < P.N || !theta_host || !ws || ((uintptr_t)ws & 255) != 0)
    return efail(p, SDF_ERR_INVALID_ARG, "diag angles: bad pointer");
  if (ws_bytes < need) return efail(p, SDF_ERR_WORKSPACE, "diag angles: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = P.N;
  const int nchunk = 2 * nsm;
  char *w = (char *)ws;
  double *Qp = (double *)w;
  w += al256(sizeof(double) * (size_t)N * k);
  double *Qv = (double *)w;
  w += al256(sizeof(double) * (size_t)N * k);
  double *T = (double *)w;
  w += al256(sizeof(double) * (size_t)N * k);
  double *part = (double *)w;
  w += al256(sizeof(double) * (size_t)nchunk * k * k);
  double *small = (double *)w;
  const unsigned grid = (unsigned)std::min<long long>((N * k + ET - 1) / ET, nsm * 8LL);
  if (dt == SDF_F64)
    k_restrict_modes<double><<<grid, ET, 0, s>>>((const double *)phi, ld, k, N, active_dev, Qp);
  else if (dt == SDF_F32)
    k_restrict_modes<float><<<grid, ET, 0, s>>>((const float *)phi, ld, k, N, active_dev, Qp);
  else
    k_restrict_modes<__nv_bfloat16><<<grid, ET, 0, s>>>((const __nv_bfloat16 *)phi, ld, k, N,
                                                         active_dev, Qp);
  ECK(cudaGetLastError());
  ECK(cudaMemcpy2DAsync(Qv, sizeof(double) * N, V_dev, sizeof(double) * ldv, sizeof(double) * N, k,
                        cudaMemcpyDeviceToDevice, s));
  BlockOps ops{p, s, N, nchunk, part, small, k};
  double *A1 = Qp, *A2 = Qv, *tmp = T;
  sdf_status e = cholqr3(ops, A1, tmp, k, false, "diag angles: restricted modes rank deficient");
  if (e != SDF_OK) return e;
  e = cholqr3(ops, A2, tmp, k, false, "diag angles: V rank deficient");
  if (e != SDF_OK) return e;
  std::vector<double> C;
  e = ops.gram(A1, A2, k, C);  // C[i][j] = q_phi,i . q_v,j
  if (e != SDF_OK) return e;
  for (int r = 1; r <= k; ++r) {
    std::vector<double> M((size_t)r * r, 0.0), wv, Vd;
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < r; ++j) {
        double t = 0.0;
        for (int q = 0; q < r; ++q) t += C[(size_t)q * k + i] * C[(size_t)q * k + j];
        M[(size_t)i * r + j] = t;
      }
    hla::jacobi_eig(r, M, wv, Vd);  // descending: wv[r - 1] = sigma_min^2
    const double c = std::sqrt(std::min(1.0, std::max(0.0, wv[r - 1])));
    theta_host[r - 1] = std::acos(c);
    // r = k: the singular values of the whole C give every principal angle
    // between the k-dimensional spans, ascending with descending sigma
    if (r == k && sorted_host)
      for (int i = 0; i < k; ++i)
        sorted_host[i] = std::acos(std::sqrt(std::min(1.0, std::max(0.0, wv[i]))));
  }
  return SDF_OK;
}

static void coarse_sizes(const sdf_problem_desc *d, int c, int nc[3], long long *Nc) {
  for (int i = 0; i < 3; ++i) nc[i] = i < d->dim ? d->n[i] / c : 1;
  *Nc = (long long)nc[0] * nc[1] * nc[2];
}

sdf_status sdf_coarse_modes_workspace_size(const sdf_problem *p, int c, int r_pool,
                                           const sdf_eig_opts *o, size_t *bytes) {
  if (!p || !o || !bytes || c < 2 || r_pool < 1 || r_pool > SDF_MAX_K) return SDF_ERR_INVALID_ARG;
  const sdf_problem_desc *d = sdf_internal_desc(p, nullptr);
  int nsm = 148, conv = 0;
  const OpParams *P = sdf_internal_op(p, &nsm, &conv);
  if (!d || !P) return SDF_ERR_INVALID_ARG;
  int nc[3];
  long long Nc;
  coarse_sizes(d, c, nc, &Nc);
  if (Nc < 2 * (long long)r_pool) return SDF_ERR_INVALID_ARG;
  sdf_problem_desc dc = *d;
  for (int i = 0; i < 3; ++i) dc.n[i] = nc[i];
  std::vector<double> kap(d->has_kappa ? Nc : 0, 1.0);
  sdf_problem *pc = nullptr;
  if (sdf_problem_create(&dc, d->has_kappa ? kap.data() : nullptr, &pc) != SDF_OK)
    return SDF_ERR_INVALID_ARG;
  size_t pb = 0;
  sdf_problem_device_bytes(pc, &pb);
  sdf_problem_destroy(pc);
  // the coarse eigensolve's own workspace: the same block layout on Nc nodes
  const int m = r_pool + (o->guard > 0 ? o->guard : std::max(16, r_pool / 2));
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const int nchunk = 2 * nsm;
  size_t eb = 4 * al(sizeof(double) * (size_t)Nc * m) + al(sizeof(double) * (size_t)nchunk * m * m) +
              al(sizeof(double) * (size_t)m * m * 2) + al(sizeof(double) * m);
  const long long N = P->N;
  size_t b = al(pb) + eb + al(sizeof(double) * (size_t)Nc * r_pool) +
             2 * al(sizeof(double) * (size_t)N * r_pool) +
             al(sizeof(double) * (size_t)nchunk * r_pool * r_pool) +
             al(sizeof(double) * (size_t)r_pool * r_pool * 2);
  *bytes = b;
  return SDF_OK;
}

sdf_status sdf_reference_modes_coarse(sdf_problem *p, int c, int r_pool, const sdf_eig_opts *o,
                                      double tau_sv, double *phi_dev, int64_t ld, int *r_out,
                                      double *lambda_c_host, sdf_eig_stats *stats, void *ws,
                                      size_t ws_bytes, void *stream) {
  if (!p) return SDF_ERR_INVALID_ARG;
  sdf_eig_opts def;
  sdf_default_eig_opts(&def);
  if (!o) o = &def;
  size_t need = 0;
  if (sdf_coarse_modes_workspace_size(p, c, r_pool, o, &need) != SDF_OK)
    return efail(p, SDF_ERR_INVALID_ARG, "coarse modes: bad factor, pool size or problem");
  int nsm = 148, conv = 0;
  const OpParams P = *sdf_internal_op(p, &nsm, &conv);
  if (conv) return efail(p, SDF_ERR_UNSUPPORTED, "coarse modes: A with convection is not symmetric");
  if (P.csr_rp) return efail(p, SDF_ERR_UNSUPPORTED, "coarse modes: no grid to coarsen");
  if (!phi_dev || ld < P.N || !ws || ((uintptr_t)ws & 255) != 0 || !(tau_sv >= 0.0))
    return efail(p, SDF_ERR_INVALID_ARG, "coarse modes: bad output, workspace or tau_sv");
  if (ws_bytes < need) return efail(p, SDF_ERR_WORKSPACE, "coarse modes: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const double *kap_f = nullptr;
  const sdf_problem_desc *d = sdf_internal_desc(p, &kap_f);
  int nc[3];
  long long Nc;
  coarse_sizes(d, c, nc, &Nc);
  // coarse problem: the same operator law, kappa injected at the nearest fine node
  sdf_problem_desc dc = *d;
  for (int i = 0; i < 3; ++i) dc.n[i] = nc[i];
  std::vector<double> kap_c;
  if (d->has_kappa) {
    kap_c.resize(Nc);
    const int nf[3] = {d->n[0], d->n[1], d->dim == 3 ? d->n[2] : 1};
    auto near = [&](int j, int m_c, int m_f) {
      int i = (int)std::lround((double)(j + 1) / (m_c + 1) * (m_f + 1)) - 1;
      return std::min(std::max(i, 0), m_f - 1);
    };
    for (int l = 0; l < nc[2]; ++l)
      for (int j = 0; j < nc[1]; ++j)
        for (int i = 0; i < nc[0]; ++i) {
          const int fi = near(i, nc[0], nf[0]), fj = near(j, nc[1], nf[1]),
                    fl = d->dim == 3 ? near(l, nc[2], nf[2]) : 0;
          kap_c[i + (size_t)nc[0] * (j + (size_t)nc[1] * l)] =
              kap_f[fi + (size_t)nf[0] * (fj + (size_t)nf[1] * fl)];
        }
  }
  sdf_problem *pc = nullptr;
  if (sdf_problem_create(&dc, d->has_kappa ? kap_c.data() : nullptr, &pc) != SDF_OK)
    return efail(p, SDF_ERR_INVALID_ARG, "coarse modes: coarse problem rejected");
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t pb = 0;
  sdf_problem_device_bytes(pc, &pb);
  char *w = (char *)ws;
  size_t off = 0;
  char *pbuf = w + off;
  off += al(pb);
  sdf_status st = sdf_problem_bind(pc, pbuf, pb, stream);
  if (st != SDF_OK) {
    sdf_problem_destroy(pc);
    return efail(p, st, "coarse modes: binding the coarse problem failed");
  }
  size_t eb = 0;
  sdf_eig_workspace_size(pc, r_pool, o, &eb);
  char *ews = w + off;
  off += al(eb);
  double *Xc = (double *)(w + off);
  off += al(sizeof(double) * (size_t)Nc * r_pool);
  double *Xf = (double *)(w + off);
  off += al(sizeof(double) * (size_t)P.N * r_pool);
  double *Xg = (double *)(w + off);
  off += al(sizeof(double) * (size_t)P.N * r_pool);
  const int nchunk = 2 * nsm;
  double *part = (double *)(w + off);
  off += al(sizeof(double) * (size_t)nchunk * r_pool * r_pool);
  double *small = (double *)(w + off);
  // 1-2. coarse eigenpairs
  std::vector<double> lam_c(r_pool);
  st = sdf_reference_modes_eig(pc, r_pool, o, Xc, Nc, lambda_c_host ? lambda_c_host : lam_c.data(),
                               nullptr, stats, ews, eb, stream);
  if (st != SDF_OK) {
    const std::string msg = std::string("coarse modes: ") + sdf_last_error(pc);
    sdf_problem_destroy(pc);
    return efail(p, st, msg.c_str());
  }
  sdf_problem_destroy(pc);
  // 3. prolongation
  k_prolong<<<dim3((unsigned)std::min<long long>((P.N + ET - 1) / ET, nsm * 4LL), r_pool), ET, 0,
              s>>>(d->dim, P.nx, P.ny, P.nz, nc[0], nc[1], nc[2], Xc, r_pool, Xf);
  ECK(cudaGetLastError());
  // 4. QR with column discard: Cholesky of the Gram matrix that skips a column
  //    whose pivot R_jj is below tau_sv times the largest column norm
  BlockOps ops{p, s, P.N, nchunk, part, small, r_pool};
  std::vector<double> G;
  st = ops.gram(Xf, Xf, r_pool, G);
  if (st != SDF_OK) return st;
  double gmax = 0.0;
  for (int j = 0; j < r_pool; ++j) gmax = std::max(gmax, G[(size_t)j * r_pool + j]);
  const double thr = tau_sv * tau_sv * gmax;
  std::vector<int> kept;
  std::vector<double> L;  // rows of the lower factor over the kept columns
  for (int j = 0; j < r_pool; ++j) {
    const int q = (int)kept.size();
    std::vector<double> row(q + 1, 0.0);
    for (int a = 0; a < q; ++a) {
      double v = G[(size_t)kept[a] * r_pool + j];
      for (int b = 0; b < a; ++b) v -= L[(size_t)a * r_pool + b] * row[b];
      row[a] = v / L[(size_t)a * r_pool + a];
    }
    double dj = G[(size_t)j * r_pool + j];
    for (int a = 0; a < q; ++a) dj -= row[a] * row[a];
    if (!(dj > thr)) continue;  // dependent column: discarded
    row[q] = std::sqrt(dj);
    L.resize((size_t)(q + 1) * r_pool, 0.0);
    for (int a = 0; a <= q; ++a) L[(size_t)q * r_pool + a] = row[a];
    kept.push_back(j);
  }
  const int rk = (int)kept.size();
  if (rk == 0) return efail(p, SDF_ERR_NOT_SPD, "coarse modes: every column discarded");
  std::vector<double> Lk((size_t)rk * rk), Wk, W((size_t)r_pool * rk, 0.0);
  for (int a = 0; a < rk; ++a)
    for (int b = 0; b <= a; ++b) Lk[(size_t)a * rk + b] = L[(size_t)a * r_pool + b];
  hla::inv_lower_transpose(rk, Lk, Wk);
  for (int a = 0; a < rk; ++a)
    for (int b = 0; b < rk; ++b) W[(size_t)kept[a] * rk + b] = Wk[(size_t)a * rk + b];
  st = ops.rotate(Xf, W, r_pool, rk, Xg);  // Xg = Xf[:, kept] R^-1
  if (st != SDF_OK) return st;
  // a second Cholesky-QR pass restores orthonormality to working precision
  std::vector<double> G2, L2, W2;
  st = ops.gram(Xg, Xg, rk, G2);
  if (st != SDF_OK) return st;
  if (!hla::cholesky(rk, G2, L2)) return efail(p, SDF_ERR_NOT_SPD, "coarse modes: QR failed");
  hla::inv_lower_transpose(rk, L2, W2);
  st = ops.rotate(Xg, W2, rk, rk, Xf);
  if (st != SDF_OK) return st;
  ECK(cudaMemcpy2DAsync(phi_dev, sizeof(double) * ld, Xf, sizeof(double) * P.N,
                        sizeof(double) * P.N, rk, cudaMemcpyDeviceToDevice, s));
  ECK(cudaStreamSynchronize(s));
  if (r_out) *r_out = rk;
  return SDF_OK;
}


}  // extern "C"
