// Gram matrices of the FP32 stage of Alg. CheFSI (Cholesky-QR step 3, Rayleigh-Ritz step 4) on the
// fifth-generation tensor cores:  G[i][j] += scale dV sum_p A[i][p] B[j][p]  per element, FP32 inputs,
// FP64 result.
//
// Precision (3xTF32): every input is split as x = x_hi + x_lo with x_hi = rn_tf32(x) and
// x_lo = rn_tf32(x - x_hi), and A B^T ~ A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T; the dropped A_lo B_lo^T
// and the rounding of x_lo leave a relative error of a few 2^-22 per product.  The tensor cores
// accumulate 64 points in FP32 in tensor memory (their additions do not round to nearest: a sum of n
// like-signed terms comes out low by up to about n 2^-25 of itself, measured 4.6e-6 at n = 512), then
// these partial sums are added into FP32 (hi, lo) pairs with an exact two-sum (Knuth), so that the sum
// over the CTA's 4096 points carries no further FP32 rounding, and the pair goes to FP64 once.  Two
// accumulator sets alternate: the sums of one period are folded while the next period's products run.
//
// One CTA of 256 threads per (element, chunk of 4096 points).  Per stage of 32 points all threads split
// the rows of A (and B) loaded one stage ahead into registers and store the four operand tiles in the
// canonical no-swizzle K-major layout (8-row x 16-byte core matrices); one thread issues the 4 K-steps x 3
// products of `tcgen05.mma.kind::tf32` (M = 128 rows of A, N = 16 * NH8 rows of B) into a tensor-memory
// accumulator and commits them to the stage's mbarrier.  Two shared-memory stages alternate, so the
// loads of stage g + 1 overlap the products of stage g.  Every wait is bounded: on time-out the kernel
// records an error and frees its tensor memory.
//
// The subspace rotation X W on the same tensor cores (k_rotate_tc) serves the exported
// dgdft_rotate_fp32; the solver's FP32 stage rotates with the CUDA-core kernel (k_linalg.cu), which
// measured faster: a 256-element sheet ALB generation took 7.57 s with it and 7.66 s with k_rotate_tc
// (loads issued a step ahead; 34 ms against 59 ms per sheet launch before that).
#include <cstdint>
#include <mutex>
#include "kernels.h"

namespace dgdft {

__device__ int g_tc_error = 0;

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcChunk = 4096;               // points per CTA
constexpr int kTcKT = 32;                    // points per stage
constexpr int kTcSub = 2;                    // stages per FP32 accumulation period (64 points)
constexpr int kTcTile = 128 * kTcKT * 4;     // bytes of one operand tile (128 rows x 32 TF32)
constexpr int kTcLBO = (128 / 8) * 128;      // bytes between K-adjacent core matrices
constexpr int kTcSBO = 128;                  // bytes between row-adjacent core matrices
constexpr int kTcCols = 256;                 // tensor-memory columns: two accumulator sets
constexpr int kTcWaitLimit = 1 << 22;

__device__ __forceinline__ int count_mode(const ElemDesc& d, int mode) {
  switch (mode) {
    case NV_BLK: return d.n_blk;
    case NV_EIG: return d.n_eig;
    case NV_ALB: return d.n_alb;
    case 4: return d.N;
    case 5: return d.NE;
    default: return 1;
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: no swizzle, K-major, start address, leading (K) and stride (row
// group) byte offsets, descriptor version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo = kTcLBO) {
  return uint64_t((addr & 0x3FFFFu) >> 4) | (uint64_t(lbo >> 4) << 16) | (uint64_t(kTcSBO >> 4) << 32) |
         (uint64_t(1) << 46);
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < kTcWaitLimit && !done; it++)
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
  return done != 0;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// 8 FP32 accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

// stores the hi and lo TF32 parts of 4 consecutive points of row i (K offset 4 kq) into the tiles
__device__ __forceinline__ void put4(unsigned char* thi, unsigned char* tlo, int i, int kq, float4 x) {
  const int off = kq * kTcLBO + (i >> 3) * kTcSBO + (i & 7) * 16;
  float4 h, l;
  h.x = tf32_rn(x.x); l.x = tf32_rn(x.x - h.x);
  h.y = tf32_rn(x.y); l.y = tf32_rn(x.y - h.y);
  h.z = tf32_rn(x.z); l.z = tf32_rn(x.z - h.z);
  h.w = tf32_rn(x.w); l.w = tf32_rn(x.w - h.w);
  *reinterpret_cast<float4*>(thi + off) = h;
  *reinterpret_cast<float4*>(tlo + off) = l;
}

__device__ __forceinline__ float4 load4(const float* row, int p, int p_end, bool vec) {
  if (vec && p + 4 <= p_end) return __ldg(reinterpret_cast<const float4*>(row + p));
  float4 x;
  x.x = p < p_end ? __ldg(row + p) : 0.f;
  x.y = p + 1 < p_end ? __ldg(row + p + 1) : 0.f;
  x.z = p + 2 < p_end ? __ldg(row + p + 2) : 0.f;
  x.w = p + 3 < p_end ? __ldg(row + p + 3) : 0.f;
  return x;
}

}  // namespace

// NH8: each thread folds 8 NH8 accumulator columns (half of N = 16 NH8)
template <int NH8>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gram_tc(BatchArgs b, const float* __restrict__ A, const long long* ao, int na_mode, const float* __restrict__ B,
              const long long* bo, int nb_mode, int npts_mode, int same, double* G, int ldg, double scale) {
  constexpr int N = 16 * NH8, NH = 8 * NH8;
  constexpr uint32_t IDESC = idesc_tf32(N);
  const int k = blockIdx.y;
  if (k >= b.M || !(b.flags == nullptr || (b.flags[k] & EF_ACTIVE))) return;
  const ElemDesc& d = b.desc[k];
  const int na = count_mode(d, na_mode), nb = count_mode(d, nb_mode), np = count_mode(d, npts_mode);
  const int p_begin = blockIdx.x * kTcChunk;
  if (p_begin >= np) return;
  const int p_end = min(np, p_begin + kTcChunk);
  extern __shared__ __align__(1024) unsigned char smem[];   // [2 stages][A_hi, A_lo, B_hi, B_lo]
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  const float* Ak = A + ao[k];
  const float* Bk = B + bo[k];
  const bool vecA = ((ao[k] | (long long)np) & 3) == 0, vecB = ((bo[k] | (long long)np) & 3) == 0;
  const int stage_bytes = (same ? 2 : 4) * kTcTile;
  float hi[NH], lo[NH];
#pragma unroll
  for (int c = 0; c < NH; c++) hi[c] = lo[c] = 0.f;
  // fold the FP32 partial sums of accumulation period p (accumulator set p & 1) into the (hi, lo) pairs
  auto fold = [&](int p) {
    fence_after();
    const uint32_t ta = tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t((p & 1) * 128 + (warp >> 2) * NH);
#pragma unroll
    for (int c = 0; c < NH8; c++) {
      float v[8];
      tmem_ld8(ta + 8 * c, v);
#pragma unroll
      for (int q = 0; q < 8; q++) {
        float& h = hi[8 * c + q];
        const float s = h + v[q], bp = s - h;
        lo[8 * c + q] += (h - (s - bp)) + (v[q] - bp);
        h = s;
      }
    }
    fence_before();
  };
  const int nst = (p_end - p_begin + kTcKT - 1) / kTcKT;
  // thread t stages row i = t % 128 at the K quads h, h + 2, h + 4, h + 6 (h = t / 128) of every stage;
  // the next stage's loads are issued as soon as this stage's values are in shared memory, so that they
  // are in flight during the barrier, the products and the folding
  const int ri = threadIdx.x & 127, rh = threadIdx.x >> 7;
  const float* Arow = Ak + (long long)ri * np;
  const float* Brow = Bk + (long long)ri * np;
  float4 xa[4], xb[4];
  auto fetch = [&](int g) {
    const int p0 = p_begin + g * kTcKT;
#pragma unroll
    for (int it = 0; it < 4; it++) {
      const int p = p0 + 4 * (rh + 2 * it);
      xa[it] = ri < na ? load4(Arow, p, p_end, vecA) : make_float4(0.f, 0.f, 0.f, 0.f);
      xb[it] = (!same && ri < nb) ? load4(Brow, p, p_end, vecB) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  fetch(0);
  bool ok = true;
  int committed = -1;   // last stage whose products were committed
  for (int g = 0; g < nst; g++) {
    const int buf = g & 1;
    unsigned char* sb = smem + buf * stage_bytes;
    // the products of stage g - 2 (same buffers) are complete
    const bool w = g < 2 || mbar_wait(smem_u32(&mbar[buf]), ((g - 2) >> 1) & 1);
    if (!__syncthreads_and(w)) { ok = false; break; }
#pragma unroll
    for (int it = 0; it < 4; it++) {
      if (ri < na) put4(sb, sb + kTcTile, ri, rh + 2 * it, xa[it]);
      if (!same && ri < nb) put4(sb + 2 * kTcTile, sb + 3 * kTcTile, ri, rh + 2 * it, xb[it]);
    }
    if (g + 1 < nst) fetch(g + 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // tiles visible to the tensor cores
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_after();
      const uint32_t acc = tmem + uint32_t(((g / kTcSub) & 1) * 128);
      const uint32_t a_hi = smem_u32(sb), a_lo = a_hi + kTcTile;
      const uint32_t b_hi = same ? a_hi : a_hi + 2 * kTcTile, b_lo = same ? a_lo : a_hi + 3 * kTcTile;
#pragma unroll
      for (int ks = 0; ks < kTcKT / 8; ks++) {
        const uint32_t o = ks * 2 * kTcLBO;   // 8 TF32 of K = two core-matrix columns
        mma_tf32(acc, smem_desc(a_hi + o), smem_desc(b_hi + o), IDESC, (g % kTcSub != 0 || ks > 0) ? 1u : 0u);
        mma_tf32(acc, smem_desc(a_hi + o), smem_desc(b_lo + o), IDESC, 1u);
        mma_tf32(acc, smem_desc(a_lo + o), smem_desc(b_hi + o), IDESC, 1u);
      }
      mma_commit(smem_u32(&mbar[buf]));
    }
    committed = g;
    if (g % kTcSub == 0 && g > 0) {
      // period g / kTcSub - 1 ended with stage g - 1; its sums are folded while stage g runs
      const bool w2 = mbar_wait(smem_u32(&mbar[(g - 1) & 1]), ((g - 1) >> 1) & 1);
      if (!__syncthreads_and(w2)) { ok = false; break; }
      fold(g / kTcSub - 1);
    }
  }
  if (ok && nst > 0) {
    const bool w3 = mbar_wait(smem_u32(&mbar[(nst - 1) & 1]), ((nst - 1) >> 1) & 1);
    if (!__syncthreads_and(w3)) ok = false;
    else fold((nst - 1) / kTcSub);
  }
  if (ok) {
    const int i = 32 * (warp & 3) + lane, j0 = (warp >> 2) * NH;
    double* Gk = G + (long long)k * ldg * ldg;
    const double f = d.dV * scale;
    if (i < na) {
#pragma unroll
      for (int c = 0; c < NH; c++)
        if (j0 + c < nb) atomicAdd(&Gk[i * ldg + j0 + c], (double(hi[c]) + double(lo[c])) * f);
    }
  } else {
    // a wait ran out: record it, let the last committed products finish (bounded), free tensor memory
    if (threadIdx.x == 0) {
      atomicExch(&g_tc_error, 1);
      if (committed >= 0) mbar_wait(smem_u32(&mbar[committed & 1]), (committed >> 1) & 1);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
  }
}


// ---- subspace rotation of FP32 blocks (Alg. CheFSI: X <- X W in Cholesky-QR and Rayleigh-Ritz) ----
// Z[j][p] = sum_i W[i][j] X[i][p] (and Z2 from X2 with the same W; with theta the squared residuals
// sum_p (Z2[j][p] - theta_j Z[j][p])^2 are added to resid2).  D[p][j] = sum_i A[p][i] B[j][i] with
// A = X^T (a tile of 128 points, K = the input vectors) and B = W^T (N = the output vectors), 3xTF32.
// One CTA per (element, 1024 points); a step is one block (X or X2) of one 128-point tile.  Steps
// alternate between two operand buffers (one when K > 80 would not fit) and the tile's accumulators
// between two tensor-memory sets, so that the loads of step s + 1 and the epilogue of tile t overlap
// the products.  Every X tile is read before any Z of its points is written: Z may alias X.
constexpr int kRotTcTiles = 8;

template <int NH8>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_rotate_tc(BatchArgs b, const float* __restrict__ X, const long long* xo, float* Z, const long long* zo,
                int nin_mode, int nout_mode, int npts_mode, const double* __restrict__ W, int ldw, const float* X2,
                float* Z2, const double* __restrict__ theta, double* resid2, int ldr, int kpad, int nbuf) {
  constexpr int N = 16 * NH8, NH = 8 * NH8;
  constexpr uint32_t IDESC = idesc_tf32(N);
  constexpr uint32_t LBO_B = (N / 8) * kTcSBO;
  const int k = blockIdx.y;
  if (k >= b.M || !(b.flags == nullptr || (b.flags[k] & EF_ACTIVE))) return;
  const ElemDesc& d = b.desc[k];
  const int nin = count_mode(d, nin_mode), nout = count_mode(d, nout_mode), np = count_mode(d, npts_mode);
  const int pc0 = blockIdx.x * kRotTcTiles * 128;
  if (pc0 >= np) return;
  const int ntile = min(kRotTcTiles, (np - pc0 + 127) / 128);
  const int nblk = X2 != nullptr ? 2 : 1;
  const int nstep = ntile * nblk;
  extern __shared__ __align__(1024) unsigned char smem[];
  // [W_hi][W_lo][nbuf x (A_hi, A_lo)]
  const int wbytes = (kpad / 4) * LBO_B, abytes = (kpad / 4) * kTcLBO;
  unsigned char* sWh = smem;
  unsigned char* sWl = smem + wbytes;
  unsigned char* sA = smem + 2 * wbytes;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ double rsum[N];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int j = threadIdx.x; j < N; j += kTcThreads) rsum[j] = 0.0;
  // W^T as the B operand (rows j < N, K = i < kpad), zero outside nout x nin
  const double* Wk = W + (long long)k * ldw * ldw;
  for (int e = threadIdx.x; e < N * kpad; e += kTcThreads) {
    const int j = e % N, i = e / N;
    const float w = (i < nin && j < nout) ? float(Wk[(long long)i * ldw + j]) : 0.f;
    const double wd = (i < nin && j < nout) ? Wk[(long long)i * ldw + j] : 0.0;
    const float h = tf32_rn(w), l = tf32_rn(float(wd - double(h)));
    const int off = (i >> 2) * LBO_B + (j >> 3) * kTcSBO + (j & 7) * 16 + (i & 3) * 4;
    *reinterpret_cast<float*>(sWh + off) = h;
    *reinterpret_cast<float*>(sWl + off) = l;
  }
  const float* Xk = X + xo[k];
  const float* X2k = X2 ? X2 + xo[k] : nullptr;
  float* Zk = Z ? Z + zo[k] : nullptr;
  float* Z2k = Z2 ? Z2 + zo[k] : nullptr;

  // A tile of step s: X (or X2) rows i < kpad at the tile's 128 points, split, K-major core matrices.
  // Thread t handles point t % 128 of the tile and the input-vector quads t / 128 + 2 it; a step's values
  // are loaded into registers (fetch) one step before they are split into shared memory (put), so the
  // loads are in flight during the products and the epilogue of the step before.
  constexpr int kMaxQ = 12;   // quads per thread at kpad = 96
  const int pp = threadIdx.x & 127, qh = threadIdx.x >> 7;
  float4 xq[kMaxQ];
  auto fetch = [&](int s) {
    const int t = s / nblk, bi = s % nblk;
    const float* src = bi ? X2k : Xk;
    const int p = pc0 + t * 128 + pp;
#pragma unroll
    for (int it = 0; it < kMaxQ; it++) {
      const int i0 = 4 * (qh + 2 * it);
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i0 < kpad && p < np) {
        if (i0 < nin) x.x = src[(long long)i0 * np + p];
        if (i0 + 1 < nin) x.y = src[(long long)(i0 + 1) * np + p];
        if (i0 + 2 < nin) x.z = src[(long long)(i0 + 2) * np + p];
        if (i0 + 3 < nin) x.w = src[(long long)(i0 + 3) * np + p];
      }
      xq[it] = x;
    }
  };
  auto put = [&](int s) {
    unsigned char* ah = sA + (s % nbuf) * 2 * abytes;
    unsigned char* al = ah + abytes;
#pragma unroll
    for (int it = 0; it < kMaxQ; it++)
      if (4 * (qh + 2 * it) < kpad) put4(ah, al, pp, qh + 2 * it, xq[it]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  };
  auto issue_step = [&](int s) {   // one thread
    const int t = s / nblk, bi = s % nblk;
    const uint32_t tm = tmem_slot + uint32_t(((t & 1) * 2 + bi) * 128);
    const uint32_t ah = smem_u32(sA + (s % nbuf) * 2 * abytes), al = ah + abytes;
    const uint32_t bh = smem_u32(sWh), bl = smem_u32(sWl);
    for (int ks = 0; ks < kpad / 8; ks++) {
      const uint32_t oa = ks * 2 * kTcLBO, ob = ks * 2 * LBO_B;
      mma_tf32(tm, smem_desc(ah + oa), smem_desc(bh + ob, LBO_B), IDESC, ks > 0 ? 1u : 0u);
      mma_tf32(tm, smem_desc(ah + oa), smem_desc(bl + ob, LBO_B), IDESC, 1u);
      mma_tf32(tm, smem_desc(al + oa), smem_desc(bh + ob, LBO_B), IDESC, 1u);
    }
    mma_commit(smem_u32(&mbar[s % nbuf]));
  };

  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  bool ok = true;
  int committed = -1, known_done = -1;   // last committed step; last step whose products were waited for
  fetch(0);
  put(0);
  fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    fence_after();
    issue_step(0);
  }
  committed = 0;
  if (nstep > 1) fetch(1);
  for (int s = 0; s < nstep && ok; s++) {
    if (s + 1 < nstep) {
      // the buffer of step s + 1 was last read by the products of step s + 1 - nbuf
      const int prev = s + 1 - nbuf;
      const bool w = prev <= known_done || mbar_wait(smem_u32(&mbar[prev % nbuf]), (prev / nbuf) & 1);
      if (!__syncthreads_and(w)) { ok = false; break; }
      known_done = max(known_done, prev);
      put(s + 1);
      if (s + 2 < nstep) fetch(s + 2);
    }
    fence_before();
    __syncthreads();
    if (s + 1 < nstep) {
      if (threadIdx.x == 0) {
        fence_after();
        issue_step(s + 1);
      }
      committed = s + 1;
    }
    if (s % nblk == nblk - 1) {
      // epilogue of tile t: the products of its steps are complete
      const int t = s / nblk;
      // (with one buffer the products of step s were already waited for before step s + 1 was loaded)
      const bool w = s <= known_done || mbar_wait(smem_u32(&mbar[s % nbuf]), (s / nbuf) & 1);
      if (!__syncthreads_and(w)) { ok = false; break; }
      known_done = s;
      fence_after();
      const int p = pc0 + t * 128 + 32 * (warp & 3) + lane;
      const uint32_t ta = tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t((t & 1) * 2 * 128 + (warp >> 2) * NH);
#pragma unroll 1
      for (int c = 0; c < NH8; c++) {
        float z[8], z2[8];
        tmem_ld8(ta + 8 * c, z);
        if (nblk == 2) tmem_ld8(ta + 128 + 8 * c, z2);
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const int j = (warp >> 2) * NH + 8 * c + q;
          const bool in = j < nout && p < np;
          if (in && Zk) Zk[(long long)j * np + p] = z[q];
          if (in && Z2k) Z2k[(long long)j * np + p] = z2[q];
          if (resid2 != nullptr && nblk == 2) {
            double e = 0.0;
            if (in) {
              const double r = double(z2[q]) - theta[(long long)k * ldr + j] * double(z[q]);
              e = r * r;
            }
            for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
            if (lane == 0 && j < nout) atomicAdd(&rsum[j], e);
          }
        }
      }
      fence_before();
    }
  }
  if (!ok && threadIdx.x == 0) {
    atomicExch(&g_tc_error, 1);
    if (committed >= 0) mbar_wait(smem_u32(&mbar[committed % nbuf]), (committed / nbuf) & 1);
  }
  fence_before();
  __syncthreads();
  if (ok && resid2 != nullptr && nblk == 2)
    for (int j = threadIdx.x; j < nout; j += kTcThreads) atomicAdd(&resid2[(long long)k * ldr + j], rsum[j]);
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// Kernel attributes are per device: set them once per device (bit per device id < 64), under a lock so
// that no host thread launches on a device before its attributes are in place.
static std::mutex g_tc_attr_mutex;
static unsigned long long g_tc_attr_devs = 0, g_rot_attr_devs = 0;
template <typename F> static void once_per_device(unsigned long long& devs, F&& set) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_tc_attr_mutex);
  const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0ull;
  if (bit && (devs & bit)) return;
  set();
  devs |= bit;
}

// Gram matrices on the tensor cores for FP32 inputs (callers zero G first).  Returns 0 when the shape is
// not handled (more than 96 rows in B or 128 in A), so that the caller falls back to the CUDA-core kernel.
int launch_gram_tc(const BatchArgs& b, const float* A, const long long* ao, int na_mode, const float* B,
                   const long long* bo, int nb_mode, int npts_mode, double* G, int ldg, cudaStream_t st,
                   double scale, int max_rows) {
  if (max_rows > 96 || max_rows <= 0) return 0;
  const int nh8 = (max_rows + 15) / 16;
  const int same = (A == B && ao == bo && na_mode == nb_mode) ? 1 : 0;
  const int sm = 2 * (same ? 2 : 4) * kTcTile;
  once_per_device(g_tc_attr_devs, [] {
    cudaFuncSetAttribute(k_gram_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4 * kTcTile);
    cudaFuncSetAttribute(k_gram_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4 * kTcTile);
    cudaFuncSetAttribute(k_gram_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4 * kTcTile);
    cudaFuncSetAttribute(k_gram_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4 * kTcTile);
    cudaFuncSetAttribute(k_gram_tc<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4 * kTcTile);
    cudaFuncSetAttribute(k_gram_tc<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4 * kTcTile);
  });
  dim3 grid((g_max_points + kTcChunk - 1) / kTcChunk, b.M);
  count_launch();
  switch (nh8) {
    case 1: k_gram_tc<1><<<grid, kTcThreads, sm, st>>>(b, A, ao, na_mode, B, bo, nb_mode, npts_mode, same, G, ldg, scale); break;
    case 2: k_gram_tc<2><<<grid, kTcThreads, sm, st>>>(b, A, ao, na_mode, B, bo, nb_mode, npts_mode, same, G, ldg, scale); break;
    case 3: k_gram_tc<3><<<grid, kTcThreads, sm, st>>>(b, A, ao, na_mode, B, bo, nb_mode, npts_mode, same, G, ldg, scale); break;
    case 4: k_gram_tc<4><<<grid, kTcThreads, sm, st>>>(b, A, ao, na_mode, B, bo, nb_mode, npts_mode, same, G, ldg, scale); break;
    case 5: k_gram_tc<5><<<grid, kTcThreads, sm, st>>>(b, A, ao, na_mode, B, bo, nb_mode, npts_mode, same, G, ldg, scale); break;
    default: k_gram_tc<6><<<grid, kTcThreads, sm, st>>>(b, A, ao, na_mode, B, bo, nb_mode, npts_mode, same, G, ldg, scale); break;
  }
  return 1;
}

// Subspace rotation of FP32 blocks on the tensor cores; 0 when the shape is not handled (more than 96
// input or output vectors), so that the caller falls back to the CUDA-core kernel.
int launch_rotate_tc(const BatchArgs& b, const float* X, const long long* xo, float* Z, const long long* zo,
                     int nin_mode, int nout_mode, int npts_mode, const double* W, int ldw, const float* X2, float* Z2,
                     const double* theta, double* resid2, int ldr, cudaStream_t st, int max_rows) {
  if (max_rows > 96 || max_rows <= 0) return 0;
  const int nh8 = (max_rows + 15) / 16, n = 16 * nh8;
  const int kpad = 8 * ((max_rows + 7) / 8);
  const int wbytes = (kpad / 4) * (n / 8) * kTcSBO, abytes = (kpad / 4) * kTcLBO;
  const int limit = 200 * 1024;
  const int nbuf = 2 * wbytes + 4 * abytes <= limit ? 2 : 1;
  const int sm = 2 * wbytes + 2 * nbuf * abytes;
  once_per_device(g_rot_attr_devs, [limit] {
    cudaFuncSetAttribute(k_rotate_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    cudaFuncSetAttribute(k_rotate_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    cudaFuncSetAttribute(k_rotate_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    cudaFuncSetAttribute(k_rotate_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    cudaFuncSetAttribute(k_rotate_tc<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    cudaFuncSetAttribute(k_rotate_tc<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
  });
  if (sm > limit) return 0;
  dim3 grid((g_max_points + kRotTcTiles * 128 - 1) / (kRotTcTiles * 128), b.M);
  count_launch();
#define DGDFT_ROT_TC(H)                                                                                        \
  k_rotate_tc<H><<<grid, kTcThreads, sm, st>>>(b, X, xo, Z, zo, nin_mode, nout_mode, npts_mode, W, ldw, X2, Z2, \
                                               theta, resid2, ldr, kpad, nbuf)
  switch (nh8) {
    case 1: DGDFT_ROT_TC(1); break;
    case 2: DGDFT_ROT_TC(2); break;
    case 3: DGDFT_ROT_TC(3); break;
    case 4: DGDFT_ROT_TC(4); break;
    case 5: DGDFT_ROT_TC(5); break;
    default: DGDFT_ROT_TC(6); break;
  }
#undef DGDFT_ROT_TC
  return 1;
}

// 1 when a tensor-core wait ran out since the last call (the flag is cleared)
int take_tc_error() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess) return 0;
  if (v) cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
  return v;
}

}  // namespace dgdft
