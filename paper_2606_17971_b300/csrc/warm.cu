// warm.cu -- the learned warm start on sm_103a: a multilayer perceptron
// mu -> POD coefficients trained and evaluated with BF16 tensor-core products
// (tcgen05.mma, FP32 accumulators in tensor memory), Adam, the POD of solved
// states, and the expansion x0 = ybar + Psi c that seeds the inner solves.
//
// The paper has no learned component; the method follows the reading stated
// in the header (include/sdf.h): POD as in Sec. 2.2.4 (mean-centred), an MLP
// with exact GELU, MSE on standardised coefficients, Adam with bias
// correction.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sdf.h"
#include "tc_device.cuh"
#include "host_linalg.h"

namespace {

thread_local std::string g_err;

sdf_status wfail(sdf_status s, const char *msg) {
  g_err = msg;
  return s;
}

#define WCK(x)                                                           \
  do {                                                                   \
    cudaError_t e_ = (x);                                                \
    if (e_ != cudaSuccess) {                                             \
      g_err = std::string(#x) + ": " + cudaGetErrorString(e_);           \
      return SDF_ERR_CUDA;                                               \
    }                                                                    \
  } while (0)

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
inline int up16(int x) { return (x + 15) & ~15; }
inline long long up128(long long x) { return (x + 127) & ~127LL; }

// ---------------------------------------------------------------------------
// tcgen05 GEMM: D (M x N) = A (M x K) * B (N x K)^T, A and B BF16 row-major
// (K contiguous, "K-major"), FP32 accumulation in tensor memory.  One CTA of
// 128 threads computes a 128-row tile for all N <= NTILE columns; K is staged
// through shared memory 64 at a time (four MMAs of K = 16).  The epilogue
// functor receives 16 consecutive accumulator columns of one row per call.
//
// Shared-memory operand layout: the no-swizzle canonical K-major layout, core
// matrices of 8 rows x 16 bytes; consecutive core matrices along K are
// LBO = 128 bytes apart, consecutive 8-row groups SBO = 1024 bytes apart.

using namespace tc;

// Error word: 1 = an MMA completion wait timed out.
template <int NTILE, class Epi>
__global__ void __launch_bounds__(GTH) k_gemm(const __nv_bfloat16 *__restrict__ A, long long lda,
                                              const __nv_bfloat16 *__restrict__ Bm, long long ldb,
                                              long long M, int N, int K, Epi epi, int *err) {
  static_assert(NTILE % 16 == 0 && NTILE >= 16 && NTILE <= 256, "N tile");
  constexpr uint32_t TCOLS = NTILE <= 32 ? 32 : (NTILE <= 64 ? 64 : (NTILE <= 128 ? 128 : 256));
  extern __shared__ __align__(1024) uint8_t dsm[];
  uint8_t *sa = dsm;                  // 128 x 64 BF16 = 16 KB
  uint8_t *sb = dsm + GM * GK * 2;    // NTILE x 64 BF16
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long m0 = (long long)blockIdx.x * GM;
  const uint32_t mb = smem_u32(&mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tbase)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(mb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  const uint32_t idesc = idesc_bf16(GM, NTILE);
  bool all_ok = true;  // every thread saw every MMA completion (CTA-uniform)
  uint32_t phase = 0;
  for (int k0 = 0; k0 < K; k0 += GK) {
    // stage A rows m0.. and B rows 0..NTILE-1, K columns k0..k0+63 (zero outside)
    for (int e = tid; e < GM * (GK / 8); e += GTH) {
      const int r = e >> 3, kg = (e & 7) * 8;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (m0 + r < M && k0 + kg < K)
        v = *reinterpret_cast<const uint4 *>(A + (m0 + r) * lda + k0 + kg);
      *reinterpret_cast<uint4 *>(sa + cm_off(r, kg)) = v;
    }
    for (int e = tid; e < NTILE * (GK / 8); e += GTH) {
      const int r = e >> 3, kg = (e & 7) * 8;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (r < N && k0 + kg < K)
        v = *reinterpret_cast<const uint4 *>(Bm + (long long)r * ldb + k0 + kg);
      *reinterpret_cast<uint4 *>(sb + cm_off(r, kg)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
#pragma unroll
      for (int s = 0; s < GK / 16; ++s) {
        if (k0 + 16 * s < K)
          tc_mma(tmem, smem_desc(a0 + s * 2 * LBO), smem_desc(b0 + s * 2 * LBO), idesc,
                 (k0 > 0 || s > 0) ? 1u : 0u);
      }
      tc_commit(mb);
    }
    // every thread waits for the MMAs before the tile is overwritten
    const bool ok = mbar_wait(mb, phase, MBAR_LIMIT);
    phase ^= 1;
    tc_fence_after();
    all_ok = __syncthreads_and(ok) != 0;
    if (!all_ok) break;
  }
  if (all_ok) {
    // epilogue: warp w owns TMEM lanes 32w .. 32w+31 = tile rows
    const long long row = m0 + warp * 32 + (tid & 31);
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < NTILE; c0 += 16) {
      float v[16];
      __syncwarp();
      tc_ld16(lane_addr + (uint32_t)c0, v);
      if (c0 < N) epi(row, c0, v);
    }
  } else if (tid == 0) {
    atomicOr(err, 1);
    // give MMAs still in flight a bounded time to land before freeing TMEM
    mbar_wait(mb, phase, MBAR_LIMIT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS)
                 : "memory");
  }
}

template <int NTILE>
constexpr size_t gemm_smem() {
  return (size_t)GM * GK * 2 + (size_t)NTILE * GK * 2;
}

__device__ __forceinline__ float gelu_f(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// ---------------------------------------------------------------------------
// Epilogues.

// forward layer: z = acc + b; Z (FP32) kept for the backward pass; hidden
// layers store g(z) in BF16 row-major (next layer's A operand) and transposed
// (the weight-gradient product's B operand); the last layer writes z to out.
struct EpiFwd {
  const float *bias;
  int nout;                  // real output width (columns >= nout are padding)
  long long mreal;           // real batch rows
  long long ldz;             // row stride of Z / Ab
  float *Z;
  __nv_bfloat16 *Ab, *At;    // hidden layers (else null)
  long long ldt;             // row stride of At (= padded batch)
  float *out;                // last layer (else null), row stride nout
  __device__ void operator()(long long row, int c0, const float v[16]) const {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int col = c0 + j;
      const bool real = col < nout && row < mreal;
      const float z = col < nout ? v[j] + bias[col] : 0.0f;
      Z[row * ldz + col] = z;
      if (Ab) {
        const float a = real ? gelu_f(z) : 0.0f;
        const __nv_bfloat16 h = __float2bfloat16_rn(a);
        Ab[row * ldz + col] = h;
        At[(long long)col * ldt + row] = h;
      } else if (real) {
        out[row * nout + col] = z;
      }
    }
  }
};

// plain FP32 store of the real block (weight gradients)
struct EpiStore {
  float *out;
  long long ld;
  long long mreal;
  int nreal;
  __device__ void operator()(long long row, int c0, const float v[16]) const {
    if (row >= mreal) return;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (c0 + j < nreal) out[row * ld + c0 + j] = v[j];
  }
};

// back-propagated error of a hidden layer: dZ = (dZ_next W) * g'(Z)
struct EpiBwd {
  const float *Z;            // pre-activation of this layer, row stride ld
  long long ld, ldt, mreal;
  int nreal;
  float *dZf;
  __nv_bfloat16 *dZb, *dZt;
  __device__ void operator()(long long row, int c0, const float v[16]) const {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int col = c0 + j;
      const bool real = col < nreal && row < mreal;
      const float d = real ? v[j] * gelu_grad_f(Z[row * ld + col]) : 0.0f;
      dZf[row * ld + col] = d;
      const __nv_bfloat16 h = __float2bfloat16_rn(d);
      dZb[row * ld + col] = h;
      dZt[(long long)col * ldt + row] = h;
    }
  }
};

// warm-start expansion: x0[b][g] = ybar[g] + acc[g][b] (rows = grid nodes,
// columns = instances)
struct EpiWarm {
  const double *ybar;
  double *x0;
  long long N;
  int B;
  __device__ void operator()(long long g, int c0, const float v[16]) const {
    if (g >= N) return;
    const double yb = ybar[g];
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (c0 + j < B) x0[(long long)(c0 + j) * N + g] = yb + (double)v[j];
  }
};

// ---------------------------------------------------------------------------
// Small kernels.

// BF16 copies of the weights: W (out x in) and W^T (in x out), zero-padded to
// multiples of 16 in both dimensions
__global__ void k_weights_bf16(const float *theta, int fin, int fout, int pin, int pout,
                               __nv_bfloat16 *Wb, __nv_bfloat16 *Wt) {
  const int n = pin * pout;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int o = e / pin, i = e % pin;
    const float w = (o < fout && i < fin) ? theta[(long long)o * fin + i] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(w);
    Wb[(long long)o * pin + i] = h;
    Wt[(long long)i * pout + o] = h;
  }
}

// inputs to BF16 (row-major and transposed), zero-padded
__global__ void k_inputs_bf16(const float *x, long long m, int fin, long long mp, int pin,
                              __nv_bfloat16 *Xb, __nv_bfloat16 *Xt) {
  const long long n = mp * pin;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / pin;
    const int i = (int)(e % pin);
    const float v = (r < m && i < fin) ? x[r * fin + i] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Xb[r * pin + i] = h;
    Xt[(long long)i * mp + r] = h;
  }
}

// MSE loss and the output layer's error dZ = 2 (y - t) / (m c); one block,
// fixed summation order
__global__ void k_mse(const float *Z, long long ld, long long m, int c, const float *t,
                      long long ldt, float *dZf, __nv_bfloat16 *dZb, __nv_bfloat16 *dZt,
                      long long mp, double *loss) {
  __shared__ double red[1024];
  double acc = 0.0;
  const double scale = 2.0 / ((double)m * c);
  for (long long e = threadIdx.x; e < mp * ld; e += blockDim.x) {
    const long long r = e / ld;
    const int j = (int)(e % ld);
    float d = 0.0f;
    if (r < m && j < c) {
      const float diff = Z[r * ld + j] - t[r * c + j];
      acc += (double)diff * (double)diff;
      d = (float)(scale * (double)diff);
    }
    dZf[r * ld + j] = d;
    const __nv_bfloat16 h = __float2bfloat16_rn(d);
    dZb[r * ld + j] = h;
    dZt[(long long)j * mp + r] = h;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / ((double)m * c);
}

// bias gradient: column sums of dZ over the real rows, one thread per column
__global__ void k_bias_grad(const float *dZf, long long ld, long long m, int nout, float *db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nout) return;
  double s = 0.0;
  for (long long r = 0; r < m; ++r) s += (double)dZf[r * ld + j];
  db[j] = (float)s;
}

__global__ void k_adam(float *theta, const float *g, float *m, float *v, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ---------------------------------------------------------------------------
// POD kernels (FP64).

__global__ void k_pod_mean(const double *Y, int m, long long N, double *ybar) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N;
       g += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += Y[(long long)i * N + g];
    ybar[g] = s / m;
  }
}

// Gram partials of the centred snapshots: part[blk][i][j] (i <= j) over the
// block's node range; a 16 x 16 tile of (i, j) per block row.
constexpr int PT = 16;
__global__ void __launch_bounds__(256) k_pod_gram(const double *Y, const double *ybar, int m,
                                                  long long N, int nchunk, double *part) {
  __shared__ double si[PT][65], sj[PT][65];
  const int ti = blockIdx.y, tj = blockIdx.z;  // tile indices (ti <= tj only)
  if (ti > tj) return;
  const int a = threadIdx.x / PT, c = threadIdx.x % PT;
  const long long per = (N + nchunk - 1) / nchunk;
  const long long g0 = blockIdx.x * per, g1 = min(N, g0 + per);
  double acc = 0.0;
  for (long long gb = g0; gb < g1; gb += 64) {
    for (int e = threadIdx.x; e < PT * 64; e += 256) {
      const int r = e / 64, k = e % 64;
      const long long g = gb + k;
      const int ii = ti * PT + r, jj = tj * PT + r;
      const double yb = g < g1 ? ybar[g] : 0.0;
      si[r][k] = (g < g1 && ii < m) ? Y[(long long)ii * N + g] - yb : 0.0;
      sj[r][k] = (g < g1 && jj < m) ? Y[(long long)jj * N + g] - yb : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 64; ++k) acc = fma(si[a][k], sj[c][k], acc);
    __syncthreads();
  }
  const int i = ti * PT + a, j = tj * PT + c;
  if (i < m && j < m) part[((long long)blockIdx.x * m + i) * m + j] = acc;
}

__global__ void k_pod_gram_reduce(const double *part, int nchunk, int m, double *C) {
  const long long n = (long long)m * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    const int a = min(i, j), b = max(i, j);
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += part[((long long)c * m + a) * m + b];
    C[e] = s;
  }
}

// Psi[g][j] = sum_i V'[i][j] (y_i - ybar)[g] with V' = V diag(1/s) (host
// supplied, m x r); Psi row-major (node-major, r contiguous) in BF16 and,
// optionally, column-major FP64
__global__ void k_pod_basis(const double *Y, const double *ybar, int m, long long N,
                            const double *Vs, int r, __nv_bfloat16 *psi_rm, double *psi_cm) {
  extern __shared__ double vs[];  // m x r
  for (int e = threadIdx.x; e < m * r; e += blockDim.x) vs[e] = Vs[e];
  __syncthreads();
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N;
       g += (long long)gridDim.x * blockDim.x) {
    double acc[SDF_POD_MAX_R];
    for (int j = 0; j < r; ++j) acc[j] = 0.0;
    const double yb = ybar[g];
    for (int i = 0; i < m; ++i) {
      const double d = Y[(long long)i * N + g] - yb;
      for (int j = 0; j < r; ++j) acc[j] = fma(vs[i * r + j], d, acc[j]);
    }
    for (int j = 0; j < r; ++j) {
      psi_rm[g * r + j] = __float2bfloat16_rn((float)acc[j]);
      if (psi_cm) psi_cm[(long long)j * N + g] = acc[j];
    }
  }
}

// per column of Psi: index of the largest |entry| (smallest index on ties),
// one block per column, then the sign of that entry
__global__ void k_pod_sign(const double *psi_cm, long long N, int *sign) {
  __shared__ double bv[256];
  __shared__ long long bi[256];
  const int j = blockIdx.x;
  double best = -1.0;
  long long bidx = 0;
  for (long long g = threadIdx.x; g < N; g += blockDim.x) {
    const double a = fabs(psi_cm[(long long)j * N + g]);
    if (a > best) {
      best = a;
      bidx = g;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      const double o = bv[threadIdx.x + s];
      const long long oi = bi[threadIdx.x + s];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) sign[j] = psi_cm[(long long)j * N + bi[0]] < 0.0 ? -1 : 1;
}

__global__ void k_pod_flip(const int *sign, long long N, int r, __nv_bfloat16 *psi_rm,
                           double *psi_cm) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * r;
       e += (long long)gridDim.x * blockDim.x) {
    const long long g = e / r;
    const int j = (int)(e % r);
    if (sign[j] < 0) {
      psi_rm[e] = __hneg(psi_rm[e]);
      psi_cm[(long long)j * N + g] = -psi_cm[(long long)j * N + g];
    }
  }
}

// POD coefficients of snapshots onto a basis: part[blk][i][j] = sum over the
// block's node range of psi_j(g) (y_i - ybar)(g), FP64, for snapshot groups of
// 16 (grid y); 16 x 16 threads: thread (a, c) holds modes a, a + 16, ... of
// snapshot c of the group.
constexpr int CT = 32;
__global__ void __launch_bounds__(256) k_pod_project(const double *Y, const double *ybar, int m,
                                                     long long N, const double *psi_cm, int r,
                                                     int nchunk, double *part) {
  __shared__ double sp[CT][SDF_POD_MAX_R + 1], sy[CT][PT + 1];
  const int a = threadIdx.x / PT, c = threadIdx.x % PT;
  const int i0 = blockIdx.y * PT;
  const long long per = (N + nchunk - 1) / nchunk;
  const long long g0 = blockIdx.x * per, g1 = min(N, g0 + per);
  constexpr int MT = SDF_POD_MAX_R / PT;
  double acc[MT];
#pragma unroll
  for (int q = 0; q < MT; ++q) acc[q] = 0.0;
  for (long long gb = g0; gb < g1; gb += CT) {
    for (int e = threadIdx.x; e < CT * SDF_POD_MAX_R; e += 256) {
      const int k = e % CT, j = e / CT;
      const long long g = gb + k;
      sp[k][j] = (g < g1 && j < r) ? psi_cm[(long long)j * N + g] : 0.0;
    }
    for (int e = threadIdx.x; e < CT * PT; e += 256) {
      const int k = e % CT, q = e / CT;
      const long long g = gb + k;
      sy[k][q] = (g < g1 && i0 + q < m) ? Y[(long long)(i0 + q) * N + g] - ybar[g] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < CT; ++k) {
      const double d = sy[k][c];
#pragma unroll
      for (int q = 0; q < MT; ++q) acc[q] = fma(sp[k][a + PT * q], d, acc[q]);
    }
    __syncthreads();
  }
  const int i = i0 + c;
  if (i < m)
#pragma unroll
    for (int q = 0; q < MT; ++q)
      if (a + PT * q < r) part[((long long)blockIdx.x * m + i) * r + a + PT * q] = acc[q];
}

// coef[i][j] = sum over blocks (in block order) of the projection partials
__global__ void k_pod_project_reduce(const double *part, int nchunk, int m, int r, double *coef) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * r; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += part[(long long)c * m * r + e];
    coef[e] = s;
  }
}

// standardised MLP outputs -> BF16 coefficients (instances x r, padded to 16
// rows) for the expansion product
__global__ void k_coef_bf16(const float *cstd, int B, int r, const float *cmean,
                            const float *cscale, int bp, __nv_bfloat16 *cb) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < bp * r; e += gridDim.x * blockDim.x) {
    const int b = e / r, j = e % r;
    const float v = b < B ? cstd[b * r + j] * cscale[j] + cmean[j] : 0.0f;
    cb[e] = __float2bfloat16_rn(v);
  }
}

// ---------------------------------------------------------------------------
// MLP workspace layout (batch m, padded rows mp = roundup(m, 128), padded
// widths p_l = roundup(width_l, 16)).

struct MlpLayout {
  int L;
  int w[SDF_MLP_MAX_LAYERS + 1], p[SDF_MLP_MAX_LAYERS + 1];
  long long mp;
  size_t wb[SDF_MLP_MAX_LAYERS], wt[SDF_MLP_MAX_LAYERS];   // BF16 W, W^T
  size_t xb[SDF_MLP_MAX_LAYERS + 1], xt[SDF_MLP_MAX_LAYERS + 1];  // BF16 A_l, A_l^T (l < L)
  size_t z[SDF_MLP_MAX_LAYERS + 1];                          // FP32 Z_l (l >= 1)
  size_t dzf[SDF_MLP_MAX_LAYERS + 1], dzb[SDF_MLP_MAX_LAYERS + 1], dzt[SDF_MLP_MAX_LAYERS + 1];
  size_t err, total;
};

bool mlp_layout(const sdf_mlp_desc *d, long long m, MlpLayout &Lo) {
  if (!d || d->n_layers < 1 || d->n_layers > SDF_MLP_MAX_LAYERS || m < 1) return false;
  Lo.L = d->n_layers;
  for (int l = 0; l <= Lo.L; ++l) {
    if (d->width[l] < 1 || d->width[l] > 256) return false;
    Lo.w[l] = d->width[l];
    Lo.p[l] = up16(d->width[l]);
  }
  Lo.mp = up128(m);
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t at = o;
    o = al256(o + b);
    return at;
  };
  for (int l = 1; l <= Lo.L; ++l) {
    Lo.wb[l - 1] = take(2ull * Lo.p[l] * Lo.p[l - 1]);
    Lo.wt[l - 1] = take(2ull * Lo.p[l] * Lo.p[l - 1]);
  }
  for (int l = 0; l < Lo.L; ++l) {
    Lo.xb[l] = take(2ull * Lo.mp * Lo.p[l]);
    Lo.xt[l] = take(2ull * Lo.mp * Lo.p[l]);
  }
  for (int l = 1; l <= Lo.L; ++l) {
    Lo.z[l] = take(4ull * Lo.mp * Lo.p[l]);
    Lo.dzf[l] = take(4ull * Lo.mp * Lo.p[l]);
    Lo.dzb[l] = take(2ull * Lo.mp * Lo.p[l]);
    Lo.dzt[l] = take(2ull * Lo.mp * Lo.p[l]);
  }
  Lo.err = take(16);
  Lo.total = o;
  return true;
}

long long param_count(const sdf_mlp_desc *d) {
  long long n = 0;
  for (int l = 1; l <= d->n_layers; ++l) n += (long long)d->width[l] * d->width[l - 1] + d->width[l];
  return n;
}

template <int NTILE, class Epi>
cudaError_t launch_gemm(const __nv_bfloat16 *A, long long lda, const __nv_bfloat16 *B,
                        long long ldb, long long M, int N, int K, const Epi &epi, int *err,
                        cudaStream_t s) {
  constexpr size_t smem = gemm_smem<NTILE>();
  // the kernel stages whole 16-element groups and hands the epilogue whole
  // 16-column groups below N
  if (M < 1 || N < 16 || N > NTILE || N % 16 != 0 || K < 16 || K % 16 != 0 || lda % 8 != 0 ||
      ldb % 8 != 0)
    return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_gemm<NTILE, Epi>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long tiles = (M + GM - 1) / GM;
  k_gemm<NTILE, Epi><<<(unsigned)tiles, GTH, smem, s>>>(A, lda, B, ldb, M, N, K, epi, err);
  return cudaGetLastError();
}

// dispatch on the padded output width
template <class Epi>
cudaError_t gemm_any(const __nv_bfloat16 *A, long long lda, const __nv_bfloat16 *B, long long ldb,
                     long long M, int N, int K, const Epi &epi, int *err, cudaStream_t s) {
  if (N <= 16) return launch_gemm<16>(A, lda, B, ldb, M, N, K, epi, err, s);
  if (N <= 32) return launch_gemm<32>(A, lda, B, ldb, M, N, K, epi, err, s);
  if (N <= 64) return launch_gemm<64>(A, lda, B, ldb, M, N, K, epi, err, s);
  if (N <= 128) return launch_gemm<128>(A, lda, B, ldb, M, N, K, epi, err, s);
  return launch_gemm<256>(A, lda, B, ldb, M, N, K, epi, err, s);
}

sdf_status check_err_word(int *err_dev, cudaStream_t s) {
  int h = 0;
  WCK(cudaMemcpyAsync(&h, err_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  WCK(cudaStreamSynchronize(s));
  if (h) return wfail(SDF_ERR_TIMEOUT, "tensor-core product: MMA completion wait timed out");
  return SDF_OK;
}

// forward pass; leaves Z_l, A_l (BF16) in the workspace
sdf_status mlp_forward_ws(const sdf_mlp_desc *d, const MlpLayout &Lo, const float *theta,
                          const float *x, long long m, float *y, char *ws, cudaStream_t s) {
  int *err = (int *)(ws + Lo.err);
  WCK(cudaMemsetAsync(err, 0, sizeof(int), s));
  long long off = 0;
  for (int l = 1; l <= Lo.L; ++l) {
    k_weights_bf16<<<64, 256, 0, s>>>(theta + off, Lo.w[l - 1], Lo.w[l], Lo.p[l - 1], Lo.p[l],
                                      (__nv_bfloat16 *)(ws + Lo.wb[l - 1]),
                                      (__nv_bfloat16 *)(ws + Lo.wt[l - 1]));
    off += (long long)Lo.w[l] * Lo.w[l - 1] + Lo.w[l];
  }
  k_inputs_bf16<<<64, 256, 0, s>>>(x, m, Lo.w[0], Lo.mp, Lo.p[0], (__nv_bfloat16 *)(ws + Lo.xb[0]),
                                   (__nv_bfloat16 *)(ws + Lo.xt[0]));
  WCK(cudaGetLastError());
  off = 0;
  for (int l = 1; l <= Lo.L; ++l) {
    const float *bias = theta + off + (long long)Lo.w[l] * Lo.w[l - 1];
    off += (long long)Lo.w[l] * Lo.w[l - 1] + Lo.w[l];
    const bool last = l == Lo.L;
    EpiFwd epi{bias,
               Lo.w[l],
               m,
               Lo.p[l],
               (float *)(ws + Lo.z[l]),
               last ? nullptr : (__nv_bfloat16 *)(ws + Lo.xb[l]),
               last ? nullptr : (__nv_bfloat16 *)(ws + Lo.xt[l]),
               Lo.mp,
               last ? y : nullptr};
    WCK(gemm_any((const __nv_bfloat16 *)(ws + Lo.xb[l - 1]), Lo.p[l - 1],
                 (const __nv_bfloat16 *)(ws + Lo.wb[l - 1]), Lo.p[l - 1], Lo.mp, Lo.p[l],
                 Lo.p[l - 1], epi, err, s));
  }
  return SDF_OK;
}

// FP64 expansion x0[b][g] = ybar[g] + sum_j psi[j][g] (cstd[b][j] cscale[j] +
// cmean[j]) with psi column-major (r x n); one block of 128 nodes stages its
// psi tile and every instance's coefficients in shared memory.
constexpr int XT = 128;
__global__ void __launch_bounds__(XT) k_warm_expand64(const double *psi, const double *ybar,
                                                      long long n, int r, const float *cstd,
                                                      const float *cmean, const float *cscale,
                                                      int B, double *x0) {
  extern __shared__ double xs[];
  double *ps = xs;                 // r x XT
  double *cs = xs + (size_t)r * XT;  // B x r
  const long long g0 = (long long)blockIdx.x * XT;
  for (int e = threadIdx.x; e < r * XT; e += XT) {
    const int j = e / XT, t = e % XT;
    ps[e] = g0 + t < n ? psi[(long long)j * n + g0 + t] : 0.0;
  }
  for (int e = threadIdx.x; e < B * r; e += XT) {
    const int j = e % r;
    cs[e] = (double)cstd[e] * (double)cscale[j] + (double)cmean[j];
  }
  __syncthreads();
  const long long g = g0 + threadIdx.x;
  if (g >= n) return;
  const double yb = ybar[g];
  for (int b = 0; b < B; ++b) {
    double acc = yb;
    for (int j = 0; j < r; ++j) acc = fma(ps[j * XT + threadIdx.x], cs[b * r + j], acc);
    x0[(long long)b * n + g] = acc;
  }
}

// instance parameters (rows of 7 doubles: a, c_x, c_y, c_z, ...) -> MLP
// inputs in [-1, 1] by min-max scaling over the parameter box
__global__ void k_scale_inputs(const double *inst, int B, int nin, const double *lo,
                               const double *hi, float *x) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * nin; e += gridDim.x * blockDim.x) {
    const int b = e / nin, i = e % nin;
    x[e] = (float)(2.0 * (inst[(long long)b * SDF_INSTANCE_DOUBLES + i] - lo[i]) / (hi[i] - lo[i]) - 1.0);
  }
}

// training targets: standardised POD coefficients (m x r, FP32)
__global__ void k_targets(const double *coef, int m, int r, const float *cmean,
                          const float *cscale, float *t) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * r; e += gridDim.x * blockDim.x) {
    const int j = e % r;
    t[e] = (float)((coef[e] - (double)cmean[j]) / (double)cscale[j]);
  }
}

// The fit's POD basis comes from the first kFitPodSnapshots snapshots (the
// method of snapshots diagonalises their Gram matrix on the host); the MLP is
// fit to the coefficients of every snapshot on that basis.
constexpr int kFitPodSnapshots = 384;
constexpr int kProjChunks = 148;

struct FitLayout {
  size_t pod_ws, psi_cm, coef, x, t, grad, am, av, loss, box, mlp_ws, ppart, total;
  size_t pod_bytes, mlp_bytes;
  int m_pod;
};

bool fit_layout(const sdf_warm_model *M, int m, FitLayout &F) {
  if (!M || m < 2 || m > SDF_FIT_MAX_SNAPSHOTS) return false;
  size_t pb = 0, mb = 0;
  F.m_pod = std::min(m, kFitPodSnapshots);
  if (sdf_pod_workspace_size(M->n, F.m_pod, &pb) != SDF_OK) return false;
  if (sdf_mlp_workspace_size(&M->mlp, m, &mb) != SDF_OK) return false;
  const long long np = param_count(&M->mlp);
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t at = o;
    o = al256(o + b);
    return at;
  };
  F.pod_ws = take(pb);
  F.psi_cm = take(sizeof(uint16_t) * (size_t)M->n * M->r);  // BF16 node-major copy
  F.coef = take(sizeof(double) * (size_t)m * M->r);
  F.x = take(sizeof(float) * (size_t)m * M->mlp.width[0]);
  F.t = take(sizeof(float) * (size_t)m * M->r);
  F.grad = take(sizeof(float) * np);
  F.am = take(sizeof(float) * np);
  F.av = take(sizeof(float) * np);
  F.loss = take(sizeof(double) * 4096);
  F.box = take(sizeof(double) * 16);
  F.mlp_ws = take(mb);
  F.ppart = take(sizeof(double) * (size_t)kProjChunks * m * M->r);
  F.total = o;
  F.pod_bytes = pb;
  F.mlp_bytes = mb;
  return true;
}

bool model_ok(const sdf_warm_model *M) {
  return M && M->theta && M->ybar && M->psi && M->cmean && M->cscale && M->n > 0 &&
         M->r >= 16 && M->r <= SDF_POD_MAX_R && M->r % 16 == 0 && M->mlp.n_layers >= 1 &&
         M->mlp.n_layers <= SDF_MLP_MAX_LAYERS && M->mlp.width[M->mlp.n_layers] == M->r &&
         M->mlp.width[0] >= 1 && M->mlp.width[0] <= 7;
}

}  // namespace

// ===========================================================================
// C ABI

extern "C" {

int64_t sdf_mlp_param_count(const sdf_mlp_desc *d) {
  if (!d || d->n_layers < 1 || d->n_layers > SDF_MLP_MAX_LAYERS) return -1;
  return param_count(d);
}

sdf_status sdf_mlp_workspace_size(const sdf_mlp_desc *d, int batch, size_t *bytes) {
  MlpLayout Lo;
  if (!bytes || !mlp_layout(d, batch, Lo))
    return wfail(SDF_ERR_INVALID_ARG, "bad MLP description or batch (widths 1..256)");
  *bytes = Lo.total;
  return SDF_OK;
}

sdf_status sdf_mlp_forward(const sdf_mlp_desc *d, const float *theta_dev, const float *x_dev,
                           int batch, float *y_dev, void *ws, size_t ws_bytes, void *stream) {
  MlpLayout Lo;
  if (!mlp_layout(d, batch, Lo)) return wfail(SDF_ERR_INVALID_ARG, "bad MLP description or batch");
  if (!theta_dev || !x_dev || !y_dev || !ws) return wfail(SDF_ERR_INVALID_ARG, "NULL pointer");
  if (((uintptr_t)ws & 255) != 0) return wfail(SDF_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  if (ws_bytes < Lo.total) return wfail(SDF_ERR_WORKSPACE, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  sdf_status st = mlp_forward_ws(d, Lo, theta_dev, x_dev, batch, y_dev, (char *)ws, s);
  if (st != SDF_OK) return st;
  return check_err_word((int *)((char *)ws + Lo.err), s);
}

sdf_status sdf_mlp_loss_grad(const sdf_mlp_desc *d, const float *theta_dev, const float *x_dev,
                             const float *t_dev, int batch, float *grad_dev, double *loss_dev,
                             void *ws, size_t ws_bytes, void *stream) {
  MlpLayout Lo;
  if (!mlp_layout(d, batch, Lo)) return wfail(SDF_ERR_INVALID_ARG, "bad MLP description or batch");
  if (!theta_dev || !x_dev || !t_dev || !grad_dev || !loss_dev || !ws)
    return wfail(SDF_ERR_INVALID_ARG, "NULL pointer");
  if (((uintptr_t)ws & 255) != 0) return wfail(SDF_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  if (ws_bytes < Lo.total) return wfail(SDF_ERR_WORKSPACE, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  char *w = (char *)ws;
  const long long m = batch;
  int *err = (int *)(w + Lo.err);
  // forward (the output layer's Z holds the predictions)
  float *yscratch = (float *)(w + Lo.dzf[Lo.L]);  // overwritten by k_mse below
  sdf_status st = mlp_forward_ws(d, Lo, theta_dev, x_dev, m, yscratch, w, s);
  if (st != SDF_OK) return st;
  const int L = Lo.L;
  k_mse<<<1, 1024, 0, s>>>((const float *)(w + Lo.z[L]), Lo.p[L], m, Lo.w[L], t_dev, Lo.w[L],
                           (float *)(w + Lo.dzf[L]), (__nv_bfloat16 *)(w + Lo.dzb[L]),
                           (__nv_bfloat16 *)(w + Lo.dzt[L]), Lo.mp, loss_dev);
  WCK(cudaGetLastError());
  // parameter offsets of each layer in theta / grad
  long long off[SDF_MLP_MAX_LAYERS + 1];
  off[1] = 0;
  for (int l = 1; l < L; ++l) off[l + 1] = off[l] + (long long)Lo.w[l] * Lo.w[l - 1] + Lo.w[l];
  for (int l = L; l >= 1; --l) {
    // dW_l = dZ_l^T A_{l-1}: M = out, N = in, K = batch
    EpiStore es{grad_dev + off[l], Lo.w[l - 1], Lo.w[l], Lo.w[l - 1]};
    WCK(gemm_any((const __nv_bfloat16 *)(w + Lo.dzt[l]), Lo.mp,
                 (const __nv_bfloat16 *)(w + Lo.xt[l - 1]), Lo.mp, Lo.p[l], Lo.p[l - 1],
                 (int)Lo.mp, es, err, s));
    k_bias_grad<<<(Lo.w[l] + 127) / 128, 128, 0, s>>>((const float *)(w + Lo.dzf[l]), Lo.p[l], m,
                                                       Lo.w[l],
                                                       grad_dev + off[l] + (long long)Lo.w[l] * Lo.w[l - 1]);
    WCK(cudaGetLastError());
    if (l > 1) {
      // dZ_{l-1} = (dZ_l W_l) * g'(Z_{l-1}): M = batch, N = in, K = out
      EpiBwd eb{(const float *)(w + Lo.z[l - 1]), Lo.p[l - 1], Lo.mp, m, Lo.w[l - 1],
                (float *)(w + Lo.dzf[l - 1]), (__nv_bfloat16 *)(w + Lo.dzb[l - 1]),
                (__nv_bfloat16 *)(w + Lo.dzt[l - 1])};
      WCK(gemm_any((const __nv_bfloat16 *)(w + Lo.dzb[l]), Lo.p[l],
                   (const __nv_bfloat16 *)(w + Lo.wt[l - 1]), Lo.p[l], Lo.mp, Lo.p[l - 1],
                   Lo.p[l], eb, err, s));
    }
  }
  return check_err_word(err, s);
}

sdf_status sdf_adam_step(float *theta_dev, const float *grad_dev, float *m_dev, float *v_dev,
                         int64_t n, int step, float lr, float beta1, float beta2, float eps,
                         void *stream) {
  if (!theta_dev || !grad_dev || !m_dev || !v_dev || n < 1 || step < 1)
    return wfail(SDF_ERR_INVALID_ARG, "bad Adam arguments");
  const float c1 = (float)(1.0 - std::pow((double)beta1, step));
  const float c2 = (float)(1.0 - std::pow((double)beta2, step));
  k_adam<<<592, 256, 0, (cudaStream_t)stream>>>(theta_dev, grad_dev, m_dev, v_dev, n, lr, beta1,
                                                 beta2, eps, c1, c2);
  WCK(cudaGetLastError());
  return SDF_OK;
}

sdf_status sdf_pod_workspace_size(int64_t n, int m, size_t *bytes) {
  if (!bytes || n < 1 || m < 2 || m > SDF_POD_MAX_SNAPSHOTS)
    return wfail(SDF_ERR_INVALID_ARG, "bad POD sizes");
  const int nchunk = 148;
  size_t o = 0;
  o = al256(o + sizeof(double) * (size_t)nchunk * m * m);  // Gram partials
  o = al256(o + sizeof(double) * (size_t)m * m);           // Gram
  o = al256(o + sizeof(double) * (size_t)m * SDF_POD_MAX_R);  // V diag(1/s)
  o = al256(o + sizeof(int) * SDF_POD_MAX_R);
  *bytes = o;
  return SDF_OK;
}

sdf_status sdf_pod(const double *Y_dev, int m, int64_t n, int r, double *ybar_dev,
                   void *psi_rm_bf16_dev, double *psi_cm_dev, double *sing_host,
                   double *coef_host, void *ws, size_t ws_bytes, void *stream) {
  size_t need = 0;
  if (sdf_pod_workspace_size(n, m, &need) != SDF_OK) return SDF_ERR_INVALID_ARG;
  if (r < 1 || r > SDF_POD_MAX_R || r > m - 1) return wfail(SDF_ERR_INVALID_ARG, "r out of range");
  if (!Y_dev || !ybar_dev || !psi_rm_bf16_dev || !psi_cm_dev || !sing_host || !ws)
    return wfail(SDF_ERR_INVALID_ARG, "NULL pointer");
  if (((uintptr_t)ws & 255) != 0) return wfail(SDF_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  if (ws_bytes < need) return wfail(SDF_ERR_WORKSPACE, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const int nchunk = 148;
  char *w = (char *)ws;
  double *part = (double *)w;
  size_t o = al256(sizeof(double) * (size_t)nchunk * m * m);
  double *C = (double *)(w + o);
  o = al256(o + sizeof(double) * (size_t)m * m);
  double *Vs = (double *)(w + o);
  o = al256(o + sizeof(double) * (size_t)m * SDF_POD_MAX_R);
  int *sign = (int *)(w + o);
  k_pod_mean<<<592, 256, 0, s>>>(Y_dev, m, n, ybar_dev);
  const int tiles = (m + PT - 1) / PT;
  k_pod_gram<<<dim3(nchunk, tiles, tiles), 256, 0, s>>>(Y_dev, ybar_dev, m, n, nchunk, part);
  k_pod_gram_reduce<<<64, 256, 0, s>>>(part, nchunk, m, C);
  WCK(cudaGetLastError());
  std::vector<double> Ch((size_t)m * m), wv, V;
  WCK(cudaMemcpyAsync(Ch.data(), C, sizeof(double) * m * m, cudaMemcpyDeviceToHost, s));
  WCK(cudaStreamSynchronize(s));
  hla::jacobi_eig(m, Ch, wv, V);
  if (!(wv[r - 1] > 0.0)) return wfail(SDF_ERR_NOT_SPD, "POD: fewer than r positive singular values");
  std::vector<double> vs((size_t)m * r);
  for (int j = 0; j < r; ++j) {
    sing_host[j] = std::sqrt(wv[j]);
    for (int i = 0; i < m; ++i) vs[(size_t)i * r + j] = V[(size_t)i * m + j] / sing_host[j];
  }
  WCK(cudaMemcpyAsync(Vs, vs.data(), sizeof(double) * m * r, cudaMemcpyHostToDevice, s));
  const size_t sm = sizeof(double) * (size_t)m * r;
  if (sm > 200 * 1024) return wfail(SDF_ERR_INVALID_ARG, "POD: m * r too large");
  WCK(cudaFuncSetAttribute(k_pod_basis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_pod_basis<<<592, 128, sm, s>>>(Y_dev, ybar_dev, m, n, Vs, r, (__nv_bfloat16 *)psi_rm_bf16_dev,
                                   psi_cm_dev);
  k_pod_sign<<<r, 256, 0, s>>>(psi_cm_dev, n, sign);
  k_pod_flip<<<592, 256, 0, s>>>(sign, n, r, (__nv_bfloat16 *)psi_rm_bf16_dev, psi_cm_dev);
  WCK(cudaGetLastError());
  std::vector<int> sg(r);
  WCK(cudaMemcpyAsync(sg.data(), sign, sizeof(int) * r, cudaMemcpyDeviceToHost, s));
  WCK(cudaStreamSynchronize(s));
  if (coef_host)
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < r; ++j)
        coef_host[(size_t)i * r + j] = sg[j] * sing_host[j] * V[(size_t)i * m + j];
  return SDF_OK;
}

sdf_status sdf_warm_expand_workspace_size(int batch, int r, size_t *bytes) {
  if (!bytes || batch < 1 || batch > 256 || r < 1 || r > SDF_POD_MAX_R)
    return wfail(SDF_ERR_INVALID_ARG, "bad sizes (batch <= 256)");
  *bytes = al256(2ull * up16(batch) * up16(r)) + 256;
  return SDF_OK;
}

sdf_status sdf_warm_expand(const void *psi_rm_bf16_dev, const double *ybar_dev, int64_t n, int r,
                           const float *cstd_dev, const float *cmean_dev, const float *cscale_dev,
                           int batch, double *x0_dev, void *ws, size_t ws_bytes, void *stream) {
  size_t need = 0;
  if (sdf_warm_expand_workspace_size(batch, r, &need) != SDF_OK) return SDF_ERR_INVALID_ARG;
  if (r % 16 != 0) return wfail(SDF_ERR_INVALID_ARG, "r must be a multiple of 16");
  if (!psi_rm_bf16_dev || !ybar_dev || !cstd_dev || !cmean_dev || !cscale_dev || !x0_dev || !ws)
    return wfail(SDF_ERR_INVALID_ARG, "NULL pointer");
  if (((uintptr_t)ws & 255) != 0 || ((uintptr_t)psi_rm_bf16_dev & 15) != 0)
    return wfail(SDF_ERR_INVALID_ARG, "workspace / Psi misaligned");
  if (ws_bytes < need) return wfail(SDF_ERR_WORKSPACE, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const int bp = up16(batch);
  __nv_bfloat16 *cb = (__nv_bfloat16 *)ws;
  int *err = (int *)((char *)ws + al256(2ull * bp * r));
  WCK(cudaMemsetAsync(err, 0, sizeof(int), s));
  k_coef_bf16<<<16, 256, 0, s>>>(cstd_dev, batch, r, cmean_dev, cscale_dev, bp, cb);
  WCK(cudaGetLastError());
  EpiWarm epi{ybar_dev, x0_dev, n, batch};
  WCK(gemm_any((const __nv_bfloat16 *)psi_rm_bf16_dev, r, cb, r, n, bp, r, epi, err, s));
  return check_err_word(err, s);
}

sdf_status sdf_warm_fit_workspace_size(const sdf_warm_model *M, int m, size_t *bytes) {
  FitLayout F;
  if (!bytes || !model_ok(M) || !fit_layout(M, m, F))
    return wfail(SDF_ERR_INVALID_ARG, "bad warm-start model or snapshot count");
  *bytes = F.total;
  return SDF_OK;
}

sdf_status sdf_warm_fit(sdf_warm_model *M, const double *Y_dev, const double *inst_dev, int m,
                        int epochs, float lr0, double *loss_host, void *ws, size_t ws_bytes,
                        void *stream) {
  FitLayout F;
  if (!model_ok(M) || !fit_layout(M, m, F))
    return wfail(SDF_ERR_INVALID_ARG, "bad warm-start model or snapshot count");
  if (!Y_dev || !inst_dev || !ws || epochs < 1 || epochs > 4096 || !(lr0 > 0.0f))
    return wfail(SDF_ERR_INVALID_ARG, "bad fit arguments");
  if (((uintptr_t)ws & 255) != 0) return wfail(SDF_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  if (ws_bytes < F.total) return wfail(SDF_ERR_WORKSPACE, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  char *w = (char *)ws;
  const int r = M->r, nin = M->mlp.width[0];
  // 1. POD of the first m_pod solved states, then the coefficients of all m
  //    states on that basis (FP64 projections)
  std::vector<double> sing(r), coef((size_t)m * r);
  sdf_status st = sdf_pod(Y_dev, F.m_pod, M->n, r, M->ybar, w + F.psi_cm, M->psi, sing.data(),
                          nullptr, w + F.pod_ws, F.pod_bytes, stream);
  if (st != SDF_OK) return st;
  k_pod_project<<<dim3(kProjChunks, (m + PT - 1) / PT), 256, 0, s>>>(
      Y_dev, M->ybar, m, M->n, M->psi, r, kProjChunks, (double *)(w + F.ppart));
  k_pod_project_reduce<<<64, 256, 0, s>>>((const double *)(w + F.ppart), kProjChunks, m, r,
                                          (double *)(w + F.coef));
  WCK(cudaGetLastError());
  WCK(cudaMemcpyAsync(coef.data(), w + F.coef, sizeof(double) * m * r, cudaMemcpyDeviceToHost, s));
  WCK(cudaStreamSynchronize(s));
  // 2. targets: coefficients centred per coefficient and divided by one common
  //    scale (the largest coefficient standard deviation), so that the loss
  //    weighs each coefficient by its share of the state
  std::vector<float> cm(r), cs(r);
  double smax = 0.0;
  for (int j = 0; j < r; ++j) {
    double mu = 0.0, var = 0.0;
    for (int i = 0; i < m; ++i) mu += coef[(size_t)i * r + j];
    mu /= m;
    for (int i = 0; i < m; ++i) {
      const double d = coef[(size_t)i * r + j] - mu;
      var += d * d;
    }
    cm[j] = (float)mu;
    smax = std::max(smax, std::sqrt(var / m));
  }
  for (int j = 0; j < r; ++j) cs[j] = (float)(smax > 0.0 ? smax : 1.0);
  WCK(cudaMemcpyAsync(M->cmean, cm.data(), sizeof(float) * r, cudaMemcpyHostToDevice, s));
  WCK(cudaMemcpyAsync(M->cscale, cs.data(), sizeof(float) * r, cudaMemcpyHostToDevice, s));
  double box[16];
  for (int i = 0; i < nin; ++i) {
    box[i] = M->in_lo[i];
    box[8 + i] = M->in_hi[i];
  }
  WCK(cudaMemcpyAsync(w + F.box, box, sizeof(box), cudaMemcpyHostToDevice, s));
  const double *lo = (const double *)(w + F.box), *hi = lo + 8;
  k_scale_inputs<<<16, 256, 0, s>>>(inst_dev, m, nin, lo, hi, (float *)(w + F.x));
  k_targets<<<64, 256, 0, s>>>((const double *)(w + F.coef), m, r, M->cmean, M->cscale,
                               (float *)(w + F.t));
  WCK(cudaGetLastError());
  // 3. full-batch Adam with cosine decay of the learning rate
  const long long np = param_count(&M->mlp);
  WCK(cudaMemsetAsync(w + F.am, 0, sizeof(float) * np, s));
  WCK(cudaMemsetAsync(w + F.av, 0, sizeof(float) * np, s));
  double *loss_dev = (double *)(w + F.loss);
  for (int ep = 1; ep <= epochs; ++ep) {
    st = sdf_mlp_loss_grad(&M->mlp, M->theta, (const float *)(w + F.x), (const float *)(w + F.t), m,
                           (float *)(w + F.grad), loss_dev + (ep - 1), w + F.mlp_ws, F.mlp_bytes,
                           stream);
    if (st != SDF_OK) return st;
    const float lr = (float)(0.5 * lr0 * (1.0 + std::cos(M_PI * (ep - 1) / (double)epochs)));
    st = sdf_adam_step(M->theta, (const float *)(w + F.grad), (float *)(w + F.am),
                       (float *)(w + F.av), np, ep, lr, 0.9f, 0.999f, 1e-8f, stream);
    if (st != SDF_OK) return st;
  }
  if (loss_host)
    WCK(cudaMemcpyAsync(loss_host, loss_dev, sizeof(double) * epochs, cudaMemcpyDeviceToHost, s));
  WCK(cudaStreamSynchronize(s));
  return SDF_OK;
}

sdf_status sdf_warm_predict_workspace_size(const sdf_warm_model *M, int batch, size_t *bytes) {
  size_t mb = 0, eb = 0;
  if (!bytes || !model_ok(M) || batch < 1 || batch > 256)
    return wfail(SDF_ERR_INVALID_ARG, "bad warm-start model or batch (<= 256)");
  if (sdf_mlp_workspace_size(&M->mlp, batch, &mb) != SDF_OK) return SDF_ERR_INVALID_ARG;
  if (sdf_warm_expand_workspace_size(batch, M->r, &eb) != SDF_OK) return SDF_ERR_INVALID_ARG;
  *bytes = al256(mb) + al256(eb) + al256(sizeof(float) * batch * (M->mlp.width[0] + M->r)) +
           al256(sizeof(double) * 16);
  return SDF_OK;
}

sdf_status sdf_warm_predict(const sdf_warm_model *M, const double *inst_dev, int batch,
                            double *x0_dev, void *ws, size_t ws_bytes, void *stream) {
  size_t need = 0;
  sdf_status st = sdf_warm_predict_workspace_size(M, batch, &need);
  if (st != SDF_OK) return st;
  if (!inst_dev || !x0_dev || !ws) return wfail(SDF_ERR_INVALID_ARG, "NULL pointer");
  if (((uintptr_t)ws & 255) != 0) return wfail(SDF_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  if (ws_bytes < need) return wfail(SDF_ERR_WORKSPACE, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  size_t mb = 0, eb = 0;
  sdf_mlp_workspace_size(&M->mlp, batch, &mb);
  sdf_warm_expand_workspace_size(batch, M->r, &eb);
  char *w = (char *)ws;
  char *mws = w, *ews = w + al256(mb);
  float *x = (float *)(ews + al256(eb));
  float *c = x + (size_t)batch * M->mlp.width[0];
  double *box = (double *)((char *)x + al256(sizeof(float) * batch * (M->mlp.width[0] + M->r)));
  const int nin = M->mlp.width[0];
  double hb[16];
  for (int i = 0; i < nin; ++i) {
    hb[i] = M->in_lo[i];
    hb[8 + i] = M->in_hi[i];
  }
  WCK(cudaMemcpyAsync(box, hb, sizeof(hb), cudaMemcpyHostToDevice, s));
  k_scale_inputs<<<4, 256, 0, s>>>(inst_dev, batch, nin, box, box + 8, x);
  WCK(cudaGetLastError());
  st = sdf_mlp_forward(&M->mlp, M->theta, x, batch, c, mws, mb, stream);
  if (st != SDF_OK) return st;
  const size_t sm = sizeof(double) * ((size_t)M->r * XT + (size_t)batch * M->r);
  WCK(cudaFuncSetAttribute(k_warm_expand64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_warm_expand64<<<(unsigned)((M->n + XT - 1) / XT), XT, sm, s>>>(
      M->psi, M->ybar, M->n, M->r, c, M->cmean, M->cscale, batch, x0_dev);
  WCK(cudaGetLastError());
  return SDF_OK;
}

const char *sdf_aux_last_error(void) { return g_err.c_str(); }

}  // extern "C"
