// eig.cu -- the reference eigensolve on sm_103a: the k smallest eigenpairs
// of A (the operator of the problem, symmetric when there is no convection),
// which are those of S = mass I + wgt A^T A with lambda_S = mass + wgt
// lambda_A^2 (Sec. 2.1.2 Eq. schur), by Chebyshev-filtered subspace iteration
// (Zhou & Saad, 2007: a scaled Chebyshev filter that damps the unwanted
// interval [a, b] of the spectrum, Rayleigh-Ritz on the filtered block).
// The paper computes its reference modes with ARPACK (Sec. 2.2.2) or in
// closed form on tensor-product grids (Sec. 2.2.8); this replaces the former.
//
// Every vector operation is FP64 on the GPU; the m x m Rayleigh-Ritz and
// Cholesky factorisations run on the host (m = k + guard <= 320).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/sdf.h"
#include "host_linalg.h"
#include "sdf_device.cuh"

// defined in sdf.cu: the operator parameters of a bound problem
const sdf::OpParams *sdf_internal_op(const sdf_problem *p, int *nsm, int *convection);
void sdf_internal_set_error(sdf_problem *p, const char *msg);

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

struct EigWs {
  double *X, *Y, *Z, *AX, *part, *small, *theta;
  int nchunk;
};

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

static int eig_block(int k, const sdf_eig_opts *o) {
  const int guard = o->guard > 0 ? o->guard : std::max(16, k / 2);
  return k + guard;
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
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t b = 4 * al(sizeof(double) * (size_t)N * m);
  b += al(sizeof(double) * (size_t)nchunk * m * m);
  b += al(sizeof(double) * (size_t)m * m * 2);
  b += al(sizeof(double) * (size_t)m);
  *bytes = b;
  return SDF_OK;
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
  const OpParams *Pp = sdf_internal_op(p, &nsm, &conv);
  const OpParams P = *Pp;
  if (conv) return efail(p, SDF_ERR_UNSUPPORTED, "eig: A with convection is not symmetric");
  if (!phi_dev || ld < P.N || !ws || ((uintptr_t)ws & 255) != 0)
    return efail(p, SDF_ERR_INVALID_ARG, "eig: bad output or workspace pointer");
  if (ws_bytes < need) return efail(p, SDF_ERR_WORKSPACE, "eig: workspace too small");
  if (o->degree < 2 || o->max_iter < 1 || !(o->tol > 0))
    return efail(p, SDF_ERR_INVALID_ARG, "eig: bad options");
  const auto t_start = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = P.N;
  const int m = eig_block(k, o);
  const int nchunk = 2 * nsm;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  char *w = (char *)ws;
  size_t off = 0;
  auto take = [&](size_t b) {
    char *at = w + off;
    off += al(b);
    return at;
  };
  double *X = (double *)take(sizeof(double) * (size_t)N * m);
  double *Y = (double *)take(sizeof(double) * (size_t)N * m);
  double *Z = (double *)take(sizeof(double) * (size_t)N * m);
  double *AX = (double *)take(sizeof(double) * (size_t)N * m);
  double *part = (double *)take(sizeof(double) * (size_t)nchunk * m * m);
  double *small = (double *)take(sizeof(double) * (size_t)m * m * 2);
  double *theta_d = (double *)take(sizeof(double) * (size_t)m);
  const int tiles = (m + GT - 1) / GT;
  const dim3 gblk((unsigned)std::min<long long>((N + ET - 1) / ET, nsm * 4LL), m);
  int64_t matvecs = 0;

  auto apply = [&](const double *Xp, const double *Xc, double *Xn, int cols, double a, double b,
                   double c) -> sdf_status {
    const dim3 g((unsigned)std::min<long long>((N + ET - 1) / ET, nsm * 4LL), cols);
    k_cheb<<<g, ET, 0, s>>>(P, Xp, Xc, Xn, N, a, b, c);
    ECK(cudaGetLastError());
    matvecs += cols;
    return SDF_OK;
  };
  // C (m x m, host) = X^T Y
  auto gram = [&](const double *Xa, const double *Ya, std::vector<double> &C) -> sdf_status {
    k_gram2<<<dim3(nchunk, tiles, tiles), 256, 0, s>>>(Xa, Ya, N, m, nchunk, part);
    k_gram2_reduce<<<64, 256, 0, s>>>(part, nchunk, m, small);
    ECK(cudaGetLastError());
    C.resize((size_t)m * m);
    ECK(cudaMemcpyAsync(C.data(), small, sizeof(double) * m * m, cudaMemcpyDeviceToHost, s));
    ECK(cudaStreamSynchronize(s));
    return SDF_OK;
  };
  // Yo = Xa W (W m x mo row-major, host), in column chunks whose m x mc
  // block of W fits in shared memory
  const int mc = std::max(8, std::min(m, (int)((160 * 1024) / (sizeof(double) * m)) / 8 * 8));
  ECK(cudaFuncSetAttribute(k_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(double) * (size_t)m * mc)));
  auto rotate = [&](const double *Xa, const std::vector<double> &W, int mo, double *Yo) -> sdf_status {
    for (int j0 = 0; j0 < mo; j0 += mc) {
      const int w = std::min(mc, mo - j0);
      std::vector<double> Wc((size_t)m * w);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < w; ++j) Wc[(size_t)i * w + j] = W[(size_t)i * mo + j0 + j];
      double *wd = small + (size_t)m * m;
      ECK(cudaMemcpyAsync(wd, Wc.data(), sizeof(double) * m * w, cudaMemcpyHostToDevice, s));
      k_rotate<<<(unsigned)((N + 127) / 128), 128, sizeof(double) * (size_t)m * w, s>>>(
          Xa, wd, N, m, w, Yo + (size_t)j0 * N);
      ECK(cudaGetLastError());
      // the host block is reused by the next chunk: wait for this copy
      ECK(cudaStreamSynchronize(s));
    }
    return SDF_OK;
  };
  // orthonormalise the columns of *A in place: shifted Cholesky-QR, then
  // Cholesky-QR twice (Fukaya et al., "shifted CholeskyQR3"); the shift
  // 11 (N m + m (m + 1)) u ||A||^2 keeps the first factorisation defined
  // however ill-conditioned the filtered block is; *tmp is scratch
  auto cholqr2 = [&](double *&A, double *&tmp) -> sdf_status {
    for (int rep = 0; rep < 3; ++rep) {
      std::vector<double> G, L, Wt;
      sdf_status e = gram(A, A, G);
      if (e != SDF_OK) return e;
      if (rep == 0) {
        double tr = 0.0;
        for (int i = 0; i < m; ++i) tr += G[(size_t)i * m + i];
        const double shift = 11.0 * ((double)N * m + (double)m * (m + 1)) * 1.1102230246251565e-16 * tr;
        for (int i = 0; i < m; ++i) G[(size_t)i * m + i] += shift;
      }
      if (!hla::cholesky(m, G, L)) return efail(p, SDF_ERR_NOT_SPD, "eig: block lost rank");
      hla::inv_lower_transpose(m, L, Wt);
      e = rotate(A, Wt, m, tmp);
      if (e != SDF_OK) return e;
      std::swap(A, tmp);
    }
    return SDF_OK;
  };
  std::vector<double> theta(m), V, H;
  // Rayleigh-Ritz on the orthonormal block *Xb: *Xb <- Xb V, AX = A Xb,
  // theta ascending
  auto rayleigh_ritz = [&](double *&Xb, double *&tmp) -> sdf_status {
    sdf_status e = apply(nullptr, Xb, AX, m, 1.0, 0.0, 0.0);
    if (e != SDF_OK) return e;
    e = gram(Xb, AX, H);
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
    e = rotate(Xb, V, m, tmp);
    if (e != SDF_OK) return e;
    std::swap(Xb, tmp);
    e = rotate(AX, V, m, tmp);  // A (Xb V) = (A Xb) V
    if (e != SDF_OK) return e;
    ECK(cudaMemcpyAsync(AX, tmp, sizeof(double) * (size_t)N * m, cudaMemcpyDeviceToDevice, s));
    return SDF_OK;
  };

  // spectrum bound
  k_gershgorin<<<nchunk, ET, 0, s>>>(P, N, part);
  ECK(cudaGetLastError());
  std::vector<double> gp(nchunk);
  ECK(cudaMemcpyAsync(gp.data(), part, sizeof(double) * nchunk, cudaMemcpyDeviceToHost, s));
  ECK(cudaStreamSynchronize(s));
  const double bmax = 1.01 * *std::max_element(gp.begin(), gp.end());

  // start block
  k_rand_block<<<nsm * 8, ET, 0, s>>>(X, N, m, o->seed);
  ECK(cudaGetLastError());
  double *Xb = X, *T1 = Y, *T2 = Z;
  sdf_status e = cholqr2(Xb, T1);
  if (e != SDF_OK) return e;
  e = rayleigh_ritz(Xb, T1);
  if (e != SDF_OK) return e;
  int it = 0, converged = 0;
  double maxrel = INFINITY;
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
    // T1 = (sigma / e) (A Xb - c Xb)
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
    e = cholqr2(Xb, T1);
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
    maxrel = 0.0;
    for (int j = 0; j < k; ++j) {
      double r2 = 0.0;
      for (int c = 0; c < nchunk; ++c) r2 += rp[(size_t)j * nchunk + c];
      rn[j] = std::sqrt(r2);
      maxrel = std::max(maxrel, rn[j] / std::fabs(theta[j]));
    }
    if (maxrel <= o->tol) {
      converged = 1;
      break;
    }
  }
  // output: the k wanted vectors (unit norm, column-major with leading dim ld)
  ECK(cudaMemcpy2DAsync(phi_dev, sizeof(double) * ld, Xb, sizeof(double) * N, sizeof(double) * N, k,
                        cudaMemcpyDeviceToDevice, s));
  ECK(cudaStreamSynchronize(s));
  for (int j = 0; j < k; ++j) {
    if (lambda_A_host) lambda_A_host[j] = theta[j];
    if (lambda_S_host) lambda_S_host[j] = P.mass + P.wgt * theta[j] * theta[j];
  }
  if (stats) {
    stats->iters = std::min(it, o->max_iter);
    stats->converged = converged;
    stats->max_rel_resid = maxrel;
    stats->matvecs = matvecs;
    stats->seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  }
  return converged ? SDF_OK : efail(p, SDF_ERR_CG_MAXIT, "eig: not converged within max_iter");
}

}  // extern "C"
