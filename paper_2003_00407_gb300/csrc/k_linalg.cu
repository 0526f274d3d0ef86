// Batched per-element dense kernels for the subspace steps of Alg. CheFSI:
// Gram matrices (Cholesky-QR step 3, Rayleigh-Ritz step 4), subspace
// rotations (step 5) with fused residual norms, and the small dense solvers
// (Cholesky + triangular inverse, symmetric eigensolver) run one CTA per
// element in shared memory.  All small matrices are FP64.
#include <algorithm>
#include <cstdio>
#include <type_traits>
#include "kernels.h"

namespace dgdft {

constexpr int kMaxN = 96;       // largest filter block handled by the small kernels

__device__ __forceinline__ int count_of(const ElemDesc& d, int mode) {
  switch (mode) {
    case 0: return d.n_blk;
    case 1: return d.n_eig;
    case 2: return d.n_alb;
    case 3: return 1;
    case 4: return d.N;
    case 5: return d.NE;
    default: return 0;
  }
}
__device__ __forceinline__ bool elem_active(const BatchArgs& b, int k) {
  return b.flags == nullptr || (b.flags[k] & EF_ACTIVE);
}

// ---------------------------------------------------------------- Gram ----
// G[i][j] += scale dV sum_p A[i][p] w[p] B[j][p] over one chunk of points per CTA.
// 16 x 16 threads, each owning an R x R register tile of the (16R)^2 outputs; the points
// stream through shared memory in tiles of kGramKT.  FP64 inputs accumulate in FP64;
// FP32 inputs accumulate kGramSub points in FP32 registers, then into FP64 accumulators.
// SYM (B is A, the same rows): only the 16 x 16 blocks on and above the diagonal are formed
// (R (R + 1) / 2 of the R^2 register blocks), and each one above it is also added at its mirror.
constexpr int kGramKT = 32;      // points per shared-memory tile
constexpr int kGramSub = 128;    // points per FP32 partial sum
constexpr int kGramChunk = 4096; // points per CTA
template <typename TI, int R, bool SYM>
__global__ void __launch_bounds__(256) k_gram(BatchArgs b, const TI* __restrict__ A, const long long* ao, int na_mode,
                                              const TI* __restrict__ B, const long long* bo, int nb_mode, int npts_mode,
                                              const double* __restrict__ w, const long long* wo, double* G, int ldg,
                                              double scale) {
  constexpr int NT = 16 * R;
  const int k = blockIdx.y;
  if (k >= b.M || !elem_active(b, k)) return;
  const ElemDesc& d = b.desc[k];
  const int na = count_of(d, na_mode), nb = count_of(d, nb_mode), np = count_of(d, npts_mode);
  const int p_begin = blockIdx.x * kGramChunk;
  if (p_begin >= np) return;
  const int p_end = min(np, p_begin + kGramChunk);
  __shared__ TI sA[kGramKT][NT + 1];
  __shared__ TI sB[kGramKT][NT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[R][R];
  TI part[R][R];
#pragma unroll
  for (int r = 0; r < R; r++)
#pragma unroll
    for (int c = 0; c < R; c++) { acc[r][c] = 0.0; part[r][c] = TI(0); }
  const TI* Ak = A + ao[k];
  const TI* Bk = B + bo[k];
  const double* wk = w ? w + wo[k] : nullptr;
  for (int p0 = p_begin; p0 < p_end; p0 += kGramKT) {
    for (int idx = threadIdx.x; idx < NT * kGramKT; idx += 256) {
      const int i = idx / kGramKT, kk = idx - i * kGramKT;
      const int p = p0 + kk;
      TI va = TI(0), vb = TI(0);
      if (p < p_end) {
        if (i < na) va = Ak[(long long)i * np + p];
        if (i < nb) {
          vb = Bk[(long long)i * np + p];
          if (wk != nullptr) vb = TI(double(vb) * wk[p]);
        }
      }
      sA[kk][i] = va;
      sB[kk][i] = vb;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kGramKT; kk++) {
      TI av[R], bv[R];
#pragma unroll
      for (int r = 0; r < R; r++) av[r] = sA[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < R; c++) bv[c] = sB[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < R; r++)
#pragma unroll
        for (int c = 0; c < R; c++)
          if (!SYM || r <= c) part[r][c] = fma(av[r], bv[c], part[r][c]);
    }
    __syncthreads();
    if (((p0 - p_begin + kGramKT) % kGramSub) == 0 || p0 + kGramKT >= p_end) {
#pragma unroll
      for (int r = 0; r < R; r++)
#pragma unroll
        for (int c = 0; c < R; c++) { acc[r][c] += double(part[r][c]); part[r][c] = TI(0); }
    }
  }
  double* Gk = G + (long long)k * ldg * ldg;
  const double f = d.dV * scale;
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int i = ty + 16 * r;
    if (i >= na) continue;
#pragma unroll
    for (int c = 0; c < R; c++) {
      if (SYM && r > c) continue;
      const int j = tx + 16 * c;
      if (j < nb) {
        atomicAdd(&Gk[i * ldg + j], acc[r][c] * f);
        if (SYM && r < c) atomicAdd(&Gk[j * ldg + i], acc[r][c] * f);
      }
    }
  }
}

// register tile for n <= 16R outputs per side
static int tile_r(int n) { return n <= 32 ? 2 : n <= 48 ? 3 : n <= 64 ? 4 : n <= 80 ? 5 : 6; }

template <typename TI>
void launch_gram(const BatchArgs& b, const TI* A, const long long* ao, int na_mode, const TI* B, const long long* bo,
                 int nb_mode, int npts_mode, const double* weight, const long long* wo, double* G, int ldg,
                 cudaStream_t st, double scale) {
  // callers zero G first
  if constexpr (std::is_same<TI, float>::value) {
    // FP32 inputs: 3xTF32 on the tensor cores (k_gram_tc.cu)
    if (weight == nullptr &&
        launch_gram_tc(b, A, ao, na_mode, B, bo, nb_mode, npts_mode, G, ldg, st, scale, std::max(g_max_nblk, g_max_nalb)))
      return;
  }
  dim3 grid((g_max_points + kGramChunk - 1) / kGramChunk, b.M);
  count_launch();
  const bool sym = A == B && ao == bo && na_mode == nb_mode;
#define DGDFT_GRAM(RR)                                                                                            \
  if (sym) k_gram<TI, RR, true><<<grid, 256, 0, st>>>(b, A, ao, na_mode, B, bo, nb_mode, npts_mode, weight, wo, G, ldg, \
                                                      scale);                                                     \
  else k_gram<TI, RR, false><<<grid, 256, 0, st>>>(b, A, ao, na_mode, B, bo, nb_mode, npts_mode, weight, wo, G, ldg,    \
                                                   scale)
  switch (tile_r(g_max_nblk)) {
    case 2: DGDFT_GRAM(2); break;
    case 3: DGDFT_GRAM(3); break;
    case 4: DGDFT_GRAM(4); break;
    case 5: DGDFT_GRAM(5); break;
    default: DGDFT_GRAM(6); break;
  }
#undef DGDFT_GRAM
}
thread_local int g_max_points = 0;

// ------------------------------------------------------------- rotation ----
// Z[j][p] = sum_i W[i][j] X[i][p] over kRotTiles tiles of 16Q points per CTA (Z may be null when
// only the residuals are wanted); W is staged
// in shared memory once per CTA and each X tile before any Z of the same points is
// written, so Z may alias X.  16 x 16 threads: thread (tx, ty) owns outputs
// j = ty + 16r (r < R) at points tx + 16q (q < Q).  With X2/Z2 the same W rotates a
// second block; with theta/resid2 the squared residuals sum_p (Z2[j][p] - theta_j Z[j][p])^2
// are accumulated per column.
constexpr int kRotTiles = 8;
template <typename TX, typename TZ, int R, int Q>
__global__ void __launch_bounds__(256) k_rotate(BatchArgs b, const TX* X, const long long* xo, TZ* Z,
                                                const long long* zo, int nin_mode, int nout_mode, int npts_mode,
                                                const double* __restrict__ W, int ldw, const TX* X2, TZ* Z2,
                                                const double* __restrict__ theta, double* resid2, int ldr) {
  constexpr int NT = 16 * R, P = 16 * Q;
  const int k = blockIdx.y;
  if (k >= b.M || !elem_active(b, k)) return;
  const ElemDesc& d = b.desc[k];
  const int nin = count_of(d, nin_mode), nout = count_of(d, nout_mode), np = count_of(d, npts_mode);
  const int pc0 = blockIdx.x * kRotTiles * P;
  if (pc0 >= np) return;
  extern __shared__ __align__(16) unsigned char smem[];
  TX* sW = reinterpret_cast<TX*>(smem);     // [nin][NT]
  TX* sX = sW + nin * NT;                   // [nin][P]
  TX* sX2 = sX + nin * P;
  const double* Wk = W + (long long)k * ldw * ldw;
  for (int idx = threadIdx.x; idx < nin * NT; idx += 256) {
    const int i = idx / NT, j = idx - i * NT;
    sW[idx] = j < nout ? TX(Wk[i * ldw + j]) : TX(0);
  }
  const TX* Xk = X + xo[k];
  const TX* X2k = X2 ? X2 + xo[k] : nullptr;
  TZ* Zk = Z ? Z + zo[k] : nullptr;
  TZ* Z2k = Z2 ? Z2 + zo[k] : nullptr;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double rsum[R];
#pragma unroll
  for (int r = 0; r < R; r++) rsum[r] = 0.0;
  for (int t = 0; t < kRotTiles; t++) {
    const int p0 = pc0 + t * P;
    if (p0 >= np) break;
    __syncthreads();   // previous tile consumed (and W staged)
    for (int idx = threadIdx.x; idx < nin * P; idx += 256) {
      const int i = idx / P, pp = idx - i * P;
      const int p = p0 + pp;
      sX[idx] = (p < np) ? Xk[(long long)i * np + p] : TX(0);
      if (X2k) sX2[idx] = (p < np) ? X2k[(long long)i * np + p] : TX(0);
    }
    __syncthreads();
    TX acc[R][Q], acc2[R][Q];
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
      for (int q = 0; q < Q; q++) { acc[r][q] = TX(0); acc2[r][q] = TX(0); }
    if (X2k) {
      for (int i = 0; i < nin; i++) {
        TX wv[R], xv[Q], xv2[Q];
#pragma unroll
        for (int r = 0; r < R; r++) wv[r] = sW[i * NT + ty + 16 * r];
#pragma unroll
        for (int q = 0; q < Q; q++) { xv[q] = sX[i * P + tx + 16 * q]; xv2[q] = sX2[i * P + tx + 16 * q]; }
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
          for (int q = 0; q < Q; q++) {
            acc[r][q] = fma(wv[r], xv[q], acc[r][q]);
            acc2[r][q] = fma(wv[r], xv2[q], acc2[r][q]);
          }
      }
    } else {
      for (int i = 0; i < nin; i++) {
        TX wv[R], xv[Q];
#pragma unroll
        for (int r = 0; r < R; r++) wv[r] = sW[i * NT + ty + 16 * r];
#pragma unroll
        for (int q = 0; q < Q; q++) xv[q] = sX[i * P + tx + 16 * q];
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
          for (int q = 0; q < Q; q++) acc[r][q] = fma(wv[r], xv[q], acc[r][q]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int j = ty + 16 * r;
      if (j >= nout) continue;
#pragma unroll
      for (int q = 0; q < Q; q++) {
        const int p = p0 + tx + 16 * q;
        if (p >= np) continue;
        if (Zk) Zk[(long long)j * np + p] = TZ(acc[r][q]);
        if (Z2k) Z2k[(long long)j * np + p] = TZ(acc2[r][q]);
        if (resid2 != nullptr) {
          const double e = double(acc2[r][q]) - theta[k * ldr + j] * double(acc[r][q]);
          rsum[r] += e * e;
        }
      }
    }
  }
  if (resid2 != nullptr) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      double v = rsum[r];
      for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);   // over tx
      const int j = ty + 16 * r;
      if (tx == 0 && j < nout) atomicAdd(&resid2[k * ldr + j], v);
    }
  }
}

template <typename TX> constexpr int rot_q() { return sizeof(TX) == 4 ? 4 : 2; }
template <typename TX, int R> constexpr int rot_smem() { return (kMaxN * 16 * R + 2 * kMaxN * 16 * rot_q<TX>()) * sizeof(TX); }

template <typename TX, typename TZ>
void launch_rotate(const BatchArgs& b, const TX* X, const long long* xo, TZ* Z, const long long* zo, int nin_mode,
                   int nout_mode, int npts_mode, const double* W, int ldw, const TX* X2, TZ* Z2, const double* theta,
                   double* resid2, int ldr, cudaStream_t st) {
  constexpr int Q = rot_q<TX>();
  const int pts = kRotTiles * 16 * Q;
  dim3 grid((g_max_points + pts - 1) / pts, b.M);

  count_launch();
#define DGDFT_ROT(RR)                                                                                      \
  k_rotate<TX, TZ, RR, Q><<<grid, 256, rot_smem<TX, RR>(), st>>>(b, X, xo, Z, zo, nin_mode, nout_mode, npts_mode, \
                                                               W, ldw, X2, Z2, theta, resid2, ldr)
  switch (tile_r(g_max_nblk)) {
    case 2: DGDFT_ROT(2); break;
    case 3: DGDFT_ROT(3); break;
    case 4: DGDFT_ROT(4); break;
    case 5: DGDFT_ROT(5); break;
    default: DGDFT_ROT(6); break;
  }
#undef DGDFT_ROT
}

// -------------------------------------------------- small dense solvers ----
// Cholesky S = U^T U of the leading n x n block of A (ld = n+1, upper triangle
// overwritten by U).  Returns false on a non-positive pivot.
__device__ bool block_cholesky(double* A, int n, int lda, double min_piv_rel) {
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < n; j++) {
    if (threadIdx.x == 0) {
      const double piv = A[j * lda + j];
      if (!(piv > min_piv_rel) || !isfinite(piv)) fail = 1;
      else A[j * lda + j] = sqrt(piv);
    }
    __syncthreads();
    if (fail) return false;
    const double dj = A[j * lda + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[j * lda + i] /= dj;
    __syncthreads();
    const int m = n - j - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int r = j + 1 + idx / m, c = j + 1 + idx % m;
      if (c >= r) A[r * lda + c] -= A[j * lda + r] * A[j * lda + c];
    }
    __syncthreads();
  }
  return true;
}

// Uinv = U^{-1} (upper), column c computed by thread c
__device__ void block_upper_inverse(const double* U, double* Ui, int n, int ld) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) Ui[(idx / n) * ld + idx % n] = 0.0;
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    Ui[c * ld + c] = 1.0 / U[c * ld + c];
    for (int r = c - 1; r >= 0; r--) {
      double s = 0.0;
      for (int l = r + 1; l <= c; l++) s += U[r * ld + l] * Ui[l * ld + c];
      Ui[r * ld + c] = -s / U[r * ld + r];
    }
  }
  __syncthreads();
}

// Shifted Cholesky-QR fallback (Fukaya et al., SIAM J. Sci. Comput. 2020): on a
// failed pivot, retry with S + s I, s growing from rel_shift * trace(S).
__device__ int chol_with_shift(const double* S, double* A, int n, int ld, double rel_shift) {
  __shared__ double tr;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; i++) t += fabs(S[i * ld + i]);
    tr = t;
  }
  __syncthreads();
  double shift = 0.0;
  for (int attempt = 0; attempt < 5; attempt++) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int i = idx / n, j = idx % n;
      A[i * ld + j] = S[i * ld + j] + (i == j ? shift : 0.0);
    }
    __syncthreads();
    if (block_cholesky(A, n, ld, 1e-300)) return attempt == 0 ? 0 : EF_CHOL_SHIFT;
    shift = (shift == 0.0 ? rel_shift : shift * 100.0) * tr;
    __syncthreads();
  }
  // last resort: diagonal scaling (recorded as a failure)
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    A[i * ld + j] = (i == j) ? sqrt(fmax(S[i * ld + i], 1e-300)) : 0.0;
  }
  __syncthreads();
  return EF_CHOL_FAIL;
}

__global__ void __launch_bounds__(256) k_chol_inv(BatchArgs b, const double* S, double* Uinv, int ld, int n_mode,
                                                  double rel_shift, int* flags) {
  const int k = blockIdx.x;
  if (!elem_active(b, k)) return;
  const int n = count_of(b.desc[k], n_mode);
  extern __shared__ __align__(16) unsigned char smem[];
  const int ls = n + 1;
  double* sS = reinterpret_cast<double*>(smem);
  double* sA = sS + n * ls;
  double* sI = sA + n * ls;
  const double* Sk = S + (long long)k * ld * ld;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    sS[i * ls + j] = 0.5 * (Sk[i * ld + j] + Sk[j * ld + i]);
  }
  __syncthreads();
  const int f = chol_with_shift(sS, sA, n, ls, rel_shift);
  if (threadIdx.x == 0 && f) atomicOr(&flags[k], f);
  block_upper_inverse(sA, sI, n, ls);
  double* Uk = Uinv + (long long)k * ld * ld;
  for (int idx = threadIdx.x; idx < ld * ld; idx += blockDim.x) {
    const int i = idx / ld, j = idx % ld;
    Uk[idx] = (i < n && j < n) ? sI[i * ls + j] : 0.0;
  }
}

void launch_chol_inv(const BatchArgs& b, const double* S, double* Uinv, int ld, int n_mode, double rel_shift,
                     int* flags, cudaStream_t st) {
  const int smem = 3 * kMaxN * (kMaxN + 1) * sizeof(double);
  count_launch(); k_chol_inv<<<b.M, 256, smem, st>>>(b, S, Uinv, ld, n_mode, rel_shift, flags);
}

// C = A B for n x n blocks in shared memory (ld = n+1); transA uses A^T.
__device__ void block_matmul(const double* A, const double* B, double* C, int n, int ld, bool transA) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    double s = 0.0;
    if (transA)
      for (int l = 0; l < n; l++) s += A[l * ld + i] * B[l * ld + j];
    else
      for (int l = 0; l < n; l++) s += A[i * ld + l] * B[l * ld + j];
    C[i * ld + j] = s;
  }
  __syncthreads();
}

// Cyclic Jacobi with the round-robin parallel ordering: n/2 disjoint rotations
// per round, n-1 rounds per sweep (Golub & Van Loan, Sec. 8.5, parallel
// Jacobi).  A (n x n, ld) is diagonalised in place, V accumulates the rotations.
__device__ int block_jacobi(double* A, double* V, int n, int ld, int max_sweeps) {
  __shared__ double cs[kMaxN / 2 + 1], sn[kMaxN / 2 + 1];
  __shared__ int pp[kMaxN / 2 + 1], qq[kMaxN / 2 + 1];
  __shared__ double off2, tot2;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) V[(idx / n) * ld + idx % n] = (idx / n == idx % n);
  const int ne = n + (n & 1);
  const int npair = ne / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; sweep++) {
    if (threadIdx.x == 0) { off2 = 0.0; tot2 = 0.0; }
    __syncthreads();
    double lo = 0.0, lt = 0.0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int i = idx / n, j = idx % n;
      const double a = A[i * ld + j];
      lt += a * a;
      if (i != j) lo += a * a;
    }
    atomicAdd(&off2, lo);
    atomicAdd(&tot2, lt);
    __syncthreads();
    if (off2 <= 1e-30 * tot2 || off2 == 0.0) break;
    for (int r = 0; r < ne - 1; r++) {
      for (int i = threadIdx.x; i < npair; i += blockDim.x) {
        int p, q;
        if (i == 0) { p = r; q = ne - 1; }
        else { p = (r + i) % (ne - 1); q = (r - i + (ne - 1)) % (ne - 1); }
        if (p > q) { int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = A[p * ld + q];
          const double app = A[p * ld + p], aqq = A[q * ld + q];
          if (apq != 0.0 && fabs(apq) > 1e-300) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        pp[i] = p; qq[i] = q; cs[i] = c; sn[i] = s;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int idx = threadIdx.x; idx < npair * n; idx += blockDim.x) {
        const int i = idx / n, col = idx % n;
        const int p = pp[i], q = qq[i];
        if (q >= n || sn[i] == 0.0) continue;
        const double a = A[p * ld + col], bq = A[q * ld + col];
        A[p * ld + col] = cs[i] * a - sn[i] * bq;
        A[q * ld + col] = sn[i] * a + cs[i] * bq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int idx = threadIdx.x; idx < npair * n; idx += blockDim.x) {
        const int i = idx / n, row = idx % n;
        const int p = pp[i], q = qq[i];
        if (q >= n || sn[i] == 0.0) continue;
        double a = A[row * ld + p], bq = A[row * ld + q];
        A[row * ld + p] = cs[i] * a - sn[i] * bq;
        A[row * ld + q] = sn[i] * a + cs[i] * bq;
        a = V[row * ld + p]; bq = V[row * ld + q];
        V[row * ld + p] = cs[i] * a - sn[i] * bq;
        V[row * ld + q] = sn[i] * a + cs[i] * bq;
      }
      __syncthreads();
    }
  }
  return sweep >= max_sweeps ? EF_JACOBI_CAP : 0;
}

// rank of the diagonal entry i in ascending (desc=false) or descending order, ties by index
__device__ __forceinline__ int diag_rank(const double* A, int n, int ld, int i, bool desc) {
  const double v = A[i * ld + i];
  int r = 0;
  for (int j = 0; j < n; j++) {
    const double u = A[j * ld + j];
    const bool before = desc ? (u > v || (u == v && j < i)) : (u < v || (u == v && j < i));
    r += before;
  }
  return r;
}

// Rayleigh-Ritz on a block Y with S2 = Y^T Y dV, G = Y^T H Y dV:
//   S2 = U^T U,  H_hat = U^{-T} G U^{-1},  H_hat V = V D,  W = U^{-1} V (ascending).
__global__ void __launch_bounds__(256) k_rr_small(BatchArgs b, const double* S2, const double* G, double* W,
                                                  double* theta, int ld, int n_mode, int* flags) {
  const int k = blockIdx.x;
  if (!elem_active(b, k)) return;
  const int n = count_of(b.desc[k], n_mode);
  const int ls = n + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  double* b1 = reinterpret_cast<double*>(smem);
  double* b2 = b1 + n * ls;
  double* b3 = b2 + n * ls;
  const double* Sk = S2 + (long long)k * ld * ld;
  const double* Gk = G + (long long)k * ld * ld;
  // b3 <- sym(S2); b1 <- U (shift fallback); b2 <- U^{-1}
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    b3[i * ls + j] = 0.5 * (Sk[i * ld + j] + Sk[j * ld + i]);
  }
  __syncthreads();
  int f = chol_with_shift(b3, b1, n, ls, 1e-14);
  block_upper_inverse(b1, b2, n, ls);
  // b1 <- sym(G); b3 <- G U^{-1}; b1 <- U^{-T} b3
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    b1[i * ls + j] = 0.5 * (Gk[i * ld + j] + Gk[j * ld + i]);
  }
  __syncthreads();
  block_matmul(b1, b2, b3, n, ls, false);
  block_matmul(b2, b3, b1, n, ls, true);
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    if (i < j) {
      const double s = 0.5 * (b1[i * ls + j] + b1[j * ls + i]);
      b1[i * ls + j] = s;
      b1[j * ls + i] = s;
    }
  }
  __syncthreads();
  f |= block_jacobi(b1, b3, n, ls, 40);
  if (threadIdx.x == 0 && f) atomicOr(&flags[k], f);
  // W[:, rank(i)] = U^{-1} V[:, i]
  double* Wk = W + (long long)k * ld * ld;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, i = idx % n;
    double s = 0.0;
    for (int l = r; l < n; l++) s += b2[r * ls + l] * b3[l * ls + i];
    Wk[r * ld + diag_rank(b1, n, ls, i, false)] = s;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) theta[k * ld + diag_rank(b1, n, ls, i, false)] = b1[i * ls + i];
}

void launch_rr_small(const BatchArgs& b, const double* S2, const double* G, double* W, double* theta, int ld,
                     int n_mode, int* flags, cudaStream_t st) {
  const int smem = 3 * kMaxN * (kMaxN + 1) * sizeof(double);
  count_launch(); k_rr_small<<<b.M, 256, smem, st>>>(b, S2, G, W, theta, ld, n_mode, flags);
}

// SVD truncation by the Gram route: G = Phi_E Phi_E^T dV = V diag(sigma^2) V^T
// (descending), C[:, j] = V[:, j] / sigma_j for j < n_alb, sing = sigma.
__global__ void __launch_bounds__(256) k_svd_small(BatchArgs b, const double* G, double* C, double* sing, int ld,
                                                   int ldc) {
  const int k = blockIdx.x;
  if (!elem_active(b, k)) return;
  const ElemDesc& d = b.desc[k];
  const int n = d.n_eig, na = d.n_alb;
  const int ls = n + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  double* A = reinterpret_cast<double*>(smem);
  double* V = A + n * ls;
  const double* Gk = G + (long long)k * ld * ld;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    A[i * ls + j] = 0.5 * (Gk[i * ld + j] + Gk[j * ld + i]);
  }
  __syncthreads();
  block_jacobi(A, V, n, ls, 40);
  double* Ck = C + (long long)k * ldc * ldc;
  for (int idx = threadIdx.x; idx < ldc * ldc; idx += blockDim.x) Ck[idx] = 0.0;
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, i = idx % n;
    const int rk = diag_rank(A, n, ls, i, true);
    if (rk < na) {
      const double s = sqrt(fmax(A[i * ls + i], 0.0));
      Ck[r * ldc + rk] = V[r * ls + i] / s;
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    sing[k * ldc + diag_rank(A, n, ls, i, true)] = sqrt(fmax(A[i * ls + i], 0.0));
}

void launch_svd_small(const BatchArgs& b, const double* G, double* C, double* sing, int ld, int ldc, cudaStream_t st) {
  const int smem = 2 * kMaxN * (kMaxN + 1) * sizeof(double);
  count_launch(); k_svd_small<<<b.M, 256, smem, st>>>(b, G, C, sing, ld, ldc);
}

int set_linalg_smem_limits() {
  int e = 0;
  e |= allow_max_smem(k_rotate<float, float, 2, 4>) | allow_max_smem(k_rotate<float, float, 3, 4>);
  e |= allow_max_smem(k_rotate<float, float, 4, 4>) | allow_max_smem(k_rotate<float, float, 5, 4>);
  e |= allow_max_smem(k_rotate<float, float, 6, 4>);
  e |= allow_max_smem(k_rotate<double, double, 2, 2>) | allow_max_smem(k_rotate<double, double, 3, 2>);
  e |= allow_max_smem(k_rotate<double, double, 4, 2>) | allow_max_smem(k_rotate<double, double, 5, 2>);
  e |= allow_max_smem(k_rotate<double, double, 6, 2>);
  e |= allow_max_smem(k_chol_inv);
  e |= allow_max_smem(k_rr_small);
  e |= allow_max_smem(k_svd_small);
  return e;
}

template void launch_gram<float>(const BatchArgs&, const float*, const long long*, int, const float*, const long long*,
                                 int, int, const double*, const long long*, double*, int, cudaStream_t, double);
template void launch_gram<double>(const BatchArgs&, const double*, const long long*, int, const double*,
                                  const long long*, int, int, const double*, const long long*, double*, int,
                                  cudaStream_t, double);
template void launch_rotate<float, float>(const BatchArgs&, const float*, const long long*, float*, const long long*,
                                          int, int, int, const double*, int, const float*, float*, const double*,
                                          double*, int, cudaStream_t);
template void launch_rotate<double, double>(const BatchArgs&, const double*, const long long*, double*,
                                            const long long*, int, int, int, const double*, int, const double*,
                                            double*, const double*, double*, int, cudaStream_t);

}  // namespace dgdft
