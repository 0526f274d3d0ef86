// Fused FP32 Chebyshev step for one vector per CTA (Eq. LocalKS, Alg. CheFSI step 2):
//   y_out = alpha (H y - c y) + beta y_prev      (or y_out = H y)
// with H y = IFFT(1/2 |G|^2 FFT(y)) + V y + sum_{I,l} gamma b <b, y>.
// The half spectrum [QZ][QY][QX/2+1] of the vector stays in shared memory for the
// whole step, so the vector is read once from HBM (plus an L2 re-read in the
// epilogue), y_prev is read once and y_out written once.
// Phases (one __syncthreads between each):
//   1 x-rows: load, projector overlaps <b, y> (from the element's compact lists of the projector
//     points), R2C along x (length QX via a complex transform of QX/2), store the row's half spectrum;
//   2 y-lines: forward transform along y;
//   3 z-lines: forward along z, kinetic multiplier, inverse along z;
//   4 y-lines: inverse along y;
//   5 x-rows: C2R, nonlocal application, V y, Chebyshev combination, store.
// Each line transform runs in registers: n = R*M with the small-radix codelets.
#include "fft.cuh"

namespace dgdft {

__constant__ float2 c_twf[kTwiddleCount];

int upload_fused_twiddles(const float2* t32) {
  return cudaMemcpyToSymbol(c_twf, t32, sizeof(float2) * kTwiddleCount) != cudaSuccess;
}

using cf = cplx<float>;

template <int N, int DIR> __device__ __forceinline__ cf twc(int m) {
  const float2 w = c_twf[twiddle_offset(N) + m];
  return cf{w.x, DIR > 0 ? -w.y : w.y};
}

__host__ __device__ constexpr int pick_m(int n) {
  return (n % 8 == 0 && n / 8 <= 8) ? 8
       : (n % 6 == 0 && n / 6 <= 8) ? 6
       : (n % 5 == 0 && n / 5 <= 8) ? 5
       : (n % 4 == 0 && n / 4 <= 8) ? 4
       : (n % 3 == 0 && n / 3 <= 8) ? 3
       : (n % 2 == 0 && n / 2 <= 8) ? 2 : 1;
}

// in-place DFT of x[0..N) (natural order) in registers: N = R*M,
// X[k1 + R k2] = sum_j2 w_M^(j2 k2) w_N^(j2 k1) sum_j1 x[M j1 + j2] w_R^(j1 k1)
template <int N, int DIR> __device__ __forceinline__ void reg_fft(cf (&x)[N]) {
  constexpr int M = pick_m(N);
  constexpr int R = N / M;
#pragma unroll
  for (int j2 = 0; j2 < M; j2++) {
    cf a[R];
#pragma unroll
    for (int j1 = 0; j1 < R; j1++) a[j1] = x[M * j1 + j2];
    dft<R, DIR, float>(a);
#pragma unroll
    for (int k1 = 0; k1 < R; k1++) x[M * k1 + j2] = (j2 * k1 == 0) ? a[k1] : cmul(a[k1], twc<N, DIR>(j2 * k1));
  }
  cf out[N];
#pragma unroll
  for (int k1 = 0; k1 < R; k1++) {
    cf b[M];
#pragma unroll
    for (int j2 = 0; j2 < M; j2++) b[j2] = x[M * k1 + j2];
    dft<M, DIR, float>(b);
#pragma unroll
    for (int k2 = 0; k2 < M; k2++) out[k1 + R * k2] = b[k2];
  }
#pragma unroll
  for (int i = 0; i < N; i++) x[i] = out[i];
}

// Length-N transforms split over a lane pair (lanes i and i+16, h = lane >> 4, so that a half-warp holds
// 16 consecutive lines: conflict-free shared accesses); each lane holds N/2 points, one exchange through
// shfl_xor 16.  Unnormalised; DIR = -1 forward, +1 inverse.
// Decimation in time: lane h holds x[2m + h] on entry and X[k + h N/2] on exit (half transforms E, O of the
// even and odd samples, X_k = E_k + w^k O_k, X_{k+N/2} = E_k - w^k O_k).
template <int N, int DIR> __device__ __forceinline__ void pair_dit(cf (&x)[N / 2], int h) {
  reg_fft<N / 2, DIR>(x);
  const float s = h ? -1.f : 1.f;
#pragma unroll
  for (int k = 0; k < N / 2; k++) {
    const cf mine = h ? cmul(x[k], twc<N, DIR>(k)) : x[k];
    const cf recv = {__shfl_xor_sync(0xffffffffu, mine.re, 16), __shfl_xor_sync(0xffffffffu, mine.im, 16)};
    x[k] = cf{fmaf(s, mine.re, recv.re), fmaf(s, mine.im, recv.im)};
  }
}
// Decimation in frequency: lane h holds x[j + h N/2] on entry and X[2m + h] on exit
// (A_j = x_j + x_{j+N/2} transforms to the even outputs, B_j = (x_j - x_{j+N/2}) w^j to the odd ones).
template <int N, int DIR> __device__ __forceinline__ void pair_dif(cf (&x)[N / 2], int h) {
  const float s = h ? -1.f : 1.f;
#pragma unroll
  for (int k = 0; k < N / 2; k++) {
    const cf mine = x[k];
    const cf recv = {__shfl_xor_sync(0xffffffffu, mine.re, 16), __shfl_xor_sync(0xffffffffu, mine.im, 16)};
    const cf t = {fmaf(s, mine.re, recv.re), fmaf(s, mine.im, recv.im)};
    x[k] = h ? cmul(t, twc<N, DIR>(k)) : t;
  }
  reg_fft<N / 2, DIR>(x);
}

struct FusedArgs {
  const ElemDesc* desc;
  const int* elems;
  const int* flags;
  const FusedAtomRec* fatoms;
  ProjList plist;
  const long long* xo;
  int nvec_mode;
  int npa;
};

// 896 threads (28 warps, at most 72 registers a thread) per SM: more resident warps hide the shared-memory
// and dependency latencies of the phases better than fewer warps with evenly filled rounds of line tasks.
// A vector is held by one CTA (CL = 1) or split by z-plane parity over a cluster of two CTAs (CL = 2), whose
// z-line phase reads and writes the peer's half through distributed shared memory.
constexpr int kFusedThreads = 896;
constexpr int kFusedMaxAtoms = 96;
constexpr int kSmemOptin = 232448;   // opt-in shared memory per block (sm_103)
constexpr int kSmemPerSM = 233472;   // shared memory per SM
constexpr int kFusedStatic = 8192;   // bound on the kernel's static shared memory

// Fused instances: (Q shape, CTAs per vector, threads per CTA).  The 32x32x48 sheet elements, small test
// boxes and the uneven-batch shapes; those whose half spectrum does not fit one CTA (40x40x48, 40x32x48,
// 32x40x48) are split over two CTAs.
#define DGDFT_FUSED_SHAPES(X)                                                                             \
  X(32, 32, 48, 1, 896) X(16, 16, 16, 1, 896) X(32, 32, 32, 1, 896) X(24, 24, 32, 1, 896)                  \
  X(24, 24, 48, 1, 896) X(40, 32, 32, 1, 896) X(32, 24, 48, 1, 896) X(24, 32, 32, 1, 896)                  \
  X(24, 40, 48, 1, 896) X(40, 24, 48, 1, 896) X(40, 40, 32, 1, 896) X(24, 40, 32, 1, 896)                  \
  X(32, 24, 32, 1, 896) X(24, 32, 48, 1, 896) X(40, 24, 32, 1, 896) X(32, 40, 32, 1, 896)                  \
  X(40, 40, 48, 2, 896) X(40, 32, 48, 2, 896) X(32, 40, 48, 2, 896)

template <int QX, int QY, int QZ, int CL> constexpr int fused_spectrum_bytes() {
  return (QX / 2 + 1) * QY * (QZ / CL) * 8;
}
template <int QX, int QY, int QZ, int CL, int NT> constexpr int fused_smem_bytes() {
  static_assert(QY % 2 == 0 && QZ % 2 == 0 && CL <= 2, "lane-pair line transforms; plane parities of a split vector");
  static_assert(kFusedThreads % NT == 0 && NT % 32 == 0, "thread count");
  static_assert(fused_spectrum_bytes<QX, QY, QZ, CL>() + kFusedStatic <= kSmemOptin, "half spectrum too large");
  static_assert((kFusedThreads / NT) * (fused_spectrum_bytes<QX, QY, QZ, CL>() + kFusedStatic + 1024) <= kSmemPerSM,
                "resident CTAs exceed the SM's shared memory");
  static_assert((QX / 2 + 1) * 2 * QY * (QZ / CL) <= 65536,
                "row layout of the CTA's planes exceeds the 16-bit point index of the lists");
  return fused_spectrum_bytes<QX, QY, QZ, CL>();
}

// ---- distributed shared memory of a CTA pair ----
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
template <class T> __device__ __forceinline__ T* peer_smem(T* p, unsigned rank) {
  unsigned long long g;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(g) : "l"(reinterpret_cast<unsigned long long>(p)), "r"(rank));
  return reinterpret_cast<T*>(g);
}

// ---- projector phases from the compact point lists ----
// List entry p of atom a: g = radial factor, w = float index in the CTA's row layout | ix << 16 | iy << 20 |
// iz << 24.  The CTA's entries (per atom: all of them, or those on the planes of its parity when the vector
// is split over a pair) are numbered atom-major; warp w takes a contiguous, equal share, lanes on consecutive
// entries, 8 entries loaded ahead.  Overlaps: per atom the moments S0 = sum g y, S_x = sum g y ix, ...
// give sum g y (d0_x + ix h_x) etc.  Application: row value += g (B0 + Bx ix + By iy + Bz iz) through
// shared atomics, with B the atom's coefficients.
struct AtomC {
  float c[4];    // gamma_l N_l^2 dV for s, px, py, pz
  float d0[3];   // displacement of the box's first point
};

__device__ __forceinline__ float small_float(unsigned v) {   // exact float of v < 2^23
  return __int_as_float(0x4B000000u | v) - 8388608.f;
}

// A vector split over a CTA pair gives CTA c the z planes of parity c, plane 2s + c at its slot s.  Float4
// index in the vector of this CTA's float4 i (row-major over its plane slots); one CTA holds the planes in
// their natural order.
template <int QX, int QY, int QZ, int CL> __device__ __forceinline__ int plane_slot4(int i, unsigned crank) {
  if (CL == 1) return i;
  constexpr int PL4 = QY * QX / 4;
  return (2 * (i / PL4) + int(crank)) * PL4 + i % PL4;
}

// hi_sel: this CTA holds the odd planes of a split vector (the second part of each atom's list)
template <bool PROJ, int NW>
__device__ __forceinline__ void nl_phase(const AtomC* atoms, const int* pt_off, const int* nlo, int nseg, bool hi_sel,
                                         long long rbase, const uint2* __restrict__ lgw, const float h[3], float* buf,
                                         float (*pacc)[4]) {
  constexpr int U = 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P = pt_off[nseg];
  const int p0 = int((long long)P * warp / NW), p1 = int((long long)P * (warp + 1) / NW);
  int sg = 0;
  while (sg < nseg && pt_off[sg + 1] <= p0) sg++;
  int pos = p0;
  while (pos < p1 && sg < nseg) {
    const int seg_end = min(p1, pt_off[sg + 1]);
    const int a = sg;
    const long long eb = rbase + (long long)a * kProjCap + (hi_sel ? nlo[a] : 0) - pt_off[sg];
    const AtomC& at = atoms[a];
    const float* c = pacc[a];
    const float B0 = c[0] + c[1] * at.d0[0] + c[2] * at.d0[1] + c[3] * at.d0[2];
    const float Bx = c[1] * h[0], By = c[2] * h[1], Bz = c[3] * h[2];
    float S0 = 0.f, S1 = 0.f, S2 = 0.f, S3 = 0.f;
    for (int pb = pos + lane; pb < seg_end; pb += 32 * U) {
      float g[U];
      unsigned w[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int p = pb + 32 * u;
        if (p < seg_end) {
          const uint2 e = __ldg(lgw + eb + p);
          g[u] = __uint_as_float(e.x);
          w[u] = e.y;
        } else {
          g[u] = 0.f;
          w[u] = 0u;
        }
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        const float fx = small_float((w[u] >> 16) & 15u), fy = small_float((w[u] >> 20) & 15u),
                    fz = small_float((w[u] >> 24) & 15u);
        const int idx = int(w[u] & 0xFFFFu);
        if (PROJ) {
          const float gy = g[u] * buf[idx];
          S0 += gy;
          S1 = fmaf(gy, fx, S1);
          S2 = fmaf(gy, fy, S2);
          S3 = fmaf(gy, fz, S3);
        } else if (g[u] != 0.f) {
          atomicAdd(buf + idx, g[u] * fmaf(Bx, fx, fmaf(By, fy, fmaf(Bz, fz, B0))));
        }
      }
    }
    if (PROJ) {
      for (int o = 16; o > 0; o >>= 1) {
        S0 += __shfl_xor_sync(0xffffffffu, S0, o);
        S1 += __shfl_xor_sync(0xffffffffu, S1, o);
        S2 += __shfl_xor_sync(0xffffffffu, S2, o);
        S3 += __shfl_xor_sync(0xffffffffu, S3, o);
      }
      // sum g y, sum g y dx, sum g y dy, sum g y dz (the coefficients are applied after the phase)
      if (lane < 4)
        atomicAdd(&pacc[a][lane], lane == 0 ? S0
                                            : lane == 1 ? fmaf(at.d0[0], S0, h[0] * S1)
                                                        : lane == 2 ? fmaf(at.d0[1], S0, h[1] * S2)
                                                                    : fmaf(at.d0[2], S0, h[2] * S3));
    }
    pos = seg_end;
    sg++;
  }
}

template <int QX, int QY, int QZ, int CL, int NT>
__global__ void __launch_bounds__(NT, kFusedThreads / NT)
    k_cheb_fused(FusedArgs a, const float* __restrict__ Y, const float* __restrict__ Yprev, float* __restrict__ Yout,
                 const float* __restrict__ V, const double* __restrict__ cheb, int cheb_stride, int out_mode) {
  constexpr int NW = NT / 32;
  constexpr int HX = QX / 2 + 1;
  constexpr int PITCH = 2 * HX;            // floats per x-row slot (real row or its half spectrum)
  constexpr int QZL = QZ / CL;             // z planes held by this CTA
  constexpr int NROW = QY * QZL;
  constexpr int NF4 = NROW * QX / 4;       // float4 of this CTA's part of the vector
  constexpr int NCOL = HX * QY;            // z lines of the half spectrum
  constexpr int NCOLL = (NCOL + CL - 1) / CL;
  const unsigned crank = CL > 1 ? cluster_rank() : 0u;
  const int k = a.elems[blockIdx.y];
  const int v = blockIdx.x / CL;
  const ElemDesc& d = a.desc[k];
  const int nv = a.nvec_mode == 0 ? d.n_blk : (a.nvec_mode == 1 ? d.n_eig : (a.nvec_mode == 2 ? d.n_alb : 1));
  // both CTAs of a pair take these exits together (same vector and element)
  if (v >= nv) return;
  if (a.flags && !(a.flags[k] & EF_ACTIVE)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  cf* S = reinterpret_cast<cf*>(smem);                               // [QZL][QY][HX]
  float* Sf = reinterpret_cast<float*>(smem);
  __shared__ AtomC atoms[kFusedMaxAtoms];
  __shared__ float pacc[kFusedMaxAtoms][4];
  __shared__ float pin[CL > 1 ? kFusedMaxAtoms : 1][4];   // the peer's partial overlaps
  __shared__ float kmul[3][kMaxLine];
  __shared__ int pt_off[kFusedMaxAtoms + 1];   // first entry of each atom's part (prefix over the CTA's atoms)
  __shared__ int nlo[kFusedMaxAtoms];          // entries of each atom on even planes (split vectors)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int na = a.npa > 0 ? d.pa_count : 0;

  // ---- prologue: atom coefficients, list lengths (cooperative copies), multiplier tables ----
  for (int i = threadIdx.x; i < na * 7; i += NT)
    (&atoms[0].c[0])[i] = __ldg(a.fatoms[d.pa_begin + i / 7].c + i % 7);
  for (int i = threadIdx.x; i < na; i += NT) {
    const int lo = __ldg(a.plist.n + 2 * (d.pa_begin + i)), hi = __ldg(a.plist.n + 2 * (d.pa_begin + i) + 1);
    nlo[i] = lo;
    pt_off[i + 1] = CL == 1 ? lo + hi : (crank ? hi : lo);
  }
  for (int i = threadIdx.x; i < 3 * kMaxLine; i += NT) {
    const int ax = i / kMaxLine, kk = i % kMaxLine;
    const int n = ax == 0 ? QX : (ax == 1 ? QY : QZ);
    const int m = kk <= n / 2 ? kk : kk - n;
    kmul[ax][kk] = kk < n ? d.kscale[ax] * float(m * m) : 0.f;
  }
  for (int i = threadIdx.x; i < kFusedMaxAtoms * 4; i += NT) (&pacc[0][0])[i] = 0.f;
  __syncthreads();
  if (threadIdx.x == 0) {   // prefix over the atoms' entry counts
    pt_off[0] = 0;
    for (int ai = 0; ai < na; ai++) pt_off[ai + 1] += pt_off[ai];
  }
  const float hh[3] = {float(d.h[0]), float(d.h[1]), float(d.h[2])};
  const long long lbase = (long long)d.pa_begin * kProjCap;
  const long long vbase = a.xo[k] + (long long)v * (QX * QY * QZ);
  const float4* y4 = reinterpret_cast<const float4*>(Y + vbase);

  // ---- phase 1a: the real vector into the row slots (coalesced float4 loads, 8 in flight per thread) ----
  {
    constexpr int NIT = (NF4 + NT - 1) / NT;
#pragma unroll
    for (int b0 = 0; b0 < NIT; b0 += 8) {
      float4 q[8];
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const int i = threadIdx.x + (b0 + u) * NT;
        if (b0 + u < NIT && i < NF4) q[u] = __ldg(y4 + plane_slot4<QX, QY, QZ, CL>(i, crank));
      }
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const int i = threadIdx.x + (b0 + u) * NT;
        if (b0 + u < NIT && i < NF4) {
          const int r = i / (QX / 4), c = i % (QX / 4);
          float2* dst = reinterpret_cast<float2*>(Sf + r * PITCH + 4 * c);
          dst[0] = make_float2(q[u].x, q[u].y);
          dst[1] = make_float2(q[u].z, q[u].w);
        }
      }
    }
  }
  __syncthreads();
  // ---- phase 1b: projector overlaps <b, y> from the real rows ----
  nl_phase<true, NW>(atoms, pt_off, nlo, na, crank != 0, lbase, a.plist.gw, hh, Sf, pacc);
  __syncthreads();
  // ---- phase 1c: R2C along x in each row slot: z = x_even + i x_odd, X_k = E_k + w^k O_k ----
  for (int r = threadIdx.x; r < NROW; r += NT) {
    cf* srow = S + (long long)r * HX;
    cf zc[QX / 2];
#pragma unroll
    for (int j = 0; j < QX / 2; j++) zc[j] = srow[j];
    reg_fft<QX / 2, -1>(zc);
#pragma unroll
    for (int kx = 0; kx <= QX / 2; kx++) {
      const cf zk = zc[kx % (QX / 2)];
      const cf zm = zc[(QX / 2 - kx) % (QX / 2)];
      const cf E = {0.5f * (zk.re + zm.re), 0.5f * (zk.im - zm.im)};
      const cf O = {0.5f * (zk.im + zm.im), -0.5f * (zk.re - zm.re)};
      srow[kx] = (kx == 0 || kx == QX / 2) ? cf{E.re + (kx == 0 ? O.re : -O.re), E.im + (kx == 0 ? O.im : -O.im)}
                                           : cadd(E, cmul(O, twc<QX, -1>(kx)));
    }
  }
  __syncthreads();
  // ---- phase 2: y lines forward (lane pairs); nonlocal coefficients ----
  for (int l0 = 0; l0 < HX * QZL; l0 += 16 * NW) {
    const int h = lane >> 4, lt = l0 + warp * 16 + (lane & 15);
    const bool ok = lt < HX * QZL;
    const int l = ok ? lt : 0;
    const int kx = l % HX, z = l / HX;
    cf* base = S + (long long)z * QY * HX + kx;
    cf q[QY / 2];
#pragma unroll
    for (int m = 0; m < QY / 2; m++) q[m] = ok ? base[(2 * m + h) * HX] : cf{0.f, 0.f};
    pair_dit<QY, -1>(q, h);
    if (ok) {
#pragma unroll
      for (int m = 0; m < QY / 2; m++) base[(m + h * (QY / 2)) * HX] = q[m];
    }
  }
  if (CL == 1) {
    if (threadIdx.x < na) {
      // c_l = gamma_l N_l^2 dV <...>: the term at a point is g (c_s + c_x dx + c_y dy + c_z dz)
      float* pa = pacc[threadIdx.x];
      const float* c = atoms[threadIdx.x].c;
      pa[0] *= c[0]; pa[1] *= c[1]; pa[2] *= c[2]; pa[3] *= c[3];
    }
    __syncthreads();
  } else {
    // this CTA's partial overlaps into the peer's pin (read after the barrier)
    float* dst = peer_smem(&pin[0][0], crank ^ 1u);
    for (int i = threadIdx.x; i < na * 4; i += NT) dst[i] = (&pacc[0][0])[i];
    cluster_barrier();
  }
  // ---- phase 3: z lines (lane pairs): forward, 1/2|G|^2 / N, inverse.  Lane h holds the planes 2m + h
  // of its line: those of CTA h when the vector is split over a pair, whose lines are shared between the
  // two CTAs ----
  {
    cf* const Sp = CL > 1 ? peer_smem(S, crank ^ 1u) : S;
    const int c0 = int(crank) * NCOLL, c1 = min(NCOL, c0 + NCOLL);
    for (int l0 = c0; l0 < c1; l0 += 16 * NW) {
      const int h = lane >> 4, lt = l0 + warp * 16 + (lane & 15);
      const bool ok = lt < c1;
      const int l = ok ? lt : c0;
      const int kx = l % HX, ky = l / HX;
      constexpr int ZS = (3 - CL) * QY * HX;   // between the planes 2m + h and 2m + 2 + h of the lane
      cf* line = (CL == 1 ? S + (long long)h * QY * HX : (h == int(crank) ? S : Sp)) + l;
      cf q[QZ / 2];
#pragma unroll
      for (int m = 0; m < QZ / 2; m++) q[m] = ok ? line[(long long)m * ZS] : cf{0.f, 0.f};
      pair_dit<QZ, -1>(q, h);   // lane h: X[m + h QZ/2]
      const float kxy = kmul[0][kx] + kmul[1][ky];
#pragma unroll
      for (int m = 0; m < QZ / 2; m++) q[m] = cscale(q[m], kxy + kmul[2][m + h * (QZ / 2)]);
      pair_dif<QZ, 1>(q, h);    // lane h: planes 2m + h
      if (ok) {
#pragma unroll
        for (int m = 0; m < QZ / 2; m++) line[(long long)m * ZS] = q[m];
      }
    }
  }
  if (CL == 1) {
    __syncthreads();
  } else {
    if (threadIdx.x < na) {
      float* pa = pacc[threadIdx.x];
      const float* c = atoms[threadIdx.x].c;
#pragma unroll
      for (int j = 0; j < 4; j++) pa[j] = (pa[j] + pin[threadIdx.x][j]) * c[j];
    }
    cluster_barrier();   // the peer's writes into this CTA's planes are complete; no remote access after this
  }
  // ---- phase 4: y lines inverse (lane pairs) ----
  for (int l0 = 0; l0 < HX * QZL; l0 += 16 * NW) {
    const int h = lane >> 4, lt = l0 + warp * 16 + (lane & 15);
    const bool ok = lt < HX * QZL;
    const int l = ok ? lt : 0;
    const int kx = l % HX, z = l / HX;
    cf* base = S + (long long)z * QY * HX + kx;
    cf q[QY / 2];
#pragma unroll
    for (int m = 0; m < QY / 2; m++) q[m] = ok ? base[(m + h * (QY / 2)) * HX] : cf{0.f, 0.f};
    pair_dif<QY, 1>(q, h);
    if (ok) {
#pragma unroll
      for (int m = 0; m < QY / 2; m++) base[(2 * m + h) * HX] = q[m];
    }
  }
  __syncthreads();
  // ---- phase 5a: C2R along x; each row slot then holds T y (real) ----
  for (int r = threadIdx.x; r < NROW; r += NT) {
    cf* srow = S + (long long)r * HX;
    cf zc[QX / 2];
#pragma unroll
    for (int k2 = 0; k2 < QX / 2; k2++) {
      // E_k + i O_k with E_k = X_k + conj X_{L/2-k}, O_k = (X_k - conj X_{L/2-k}) w^{-k}
      const cf xk = srow[k2], xm = srow[QX / 2 - k2];
      const cf E = {xk.re + xm.re, xk.im - xm.im};
      const cf Dd = {xk.re - xm.re, xk.im + xm.im};
      const cf O = k2 == 0 ? Dd : cmul(Dd, twc<QX, 1>(k2));
      zc[k2] = cf{E.re - O.im, E.im + O.re};
    }
    reg_fft<QX / 2, 1>(zc);
#pragma unroll
    for (int j = 0; j < QX / 2; j++) srow[j] = zc[j];
  }
  __syncthreads();
  // ---- phase 5b: nonlocal application (shared atomics) ----
  nl_phase<false, NW>(atoms, pt_off, nlo, na, crank != 0, lbase, a.plist.gw, hh, Sf, pacc);
  __syncthreads();
  // ---- phase 5c: V y, Chebyshev combination, store (coalesced float4) ----
  float alpha = 1.f, shift = 0.f, beta = 0.f;
  if (out_mode == OUT_CHEB) {
    alpha = float(__ldg(cheb + (long long)k * cheb_stride));
    shift = float(__ldg(cheb + (long long)k * cheb_stride + 1));
    beta = float(__ldg(cheb + (long long)k * cheb_stride + 2));
  }
  const float4* v4 = reinterpret_cast<const float4*>(V + d.voff);
  const float4* p4 = (out_mode == OUT_CHEB && Yprev != nullptr && beta != 0.f)
                         ? reinterpret_cast<const float4*>(Yprev + vbase) : nullptr;
  float4* o4 = reinterpret_cast<float4*>(Yout + vbase);
  {
    // 4 chunks in flight per thread: y and V (L2), y_prev (HBM), then the combination and the store
    constexpr int NIT = (NF4 + NT - 1) / NT;
#pragma unroll
    for (int b0 = 0; b0 < NIT; b0 += 4) {
      float4 yy[4], vv[4], pp[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int i = threadIdx.x + (b0 + u) * NT;
        if (b0 + u < NIT && i < NF4) {
          const int gi = plane_slot4<QX, QY, QZ, CL>(i, crank);
          yy[u] = __ldg(y4 + gi);
          vv[u] = __ldg(v4 + gi);
          pp[u] = p4 != nullptr ? __ldg(p4 + gi) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int i = threadIdx.x + (b0 + u) * NT;
        if (b0 + u < NIT && i < NF4) {
          const int r = i / (QX / 4), c = i % (QX / 4);
          const float2* tr = reinterpret_cast<const float2*>(Sf + r * PITCH + 4 * c);
          const float2 t0 = tr[0], t1 = tr[1];
          float4 h = {t0.x + vv[u].x * yy[u].x, t0.y + vv[u].y * yy[u].y, t1.x + vv[u].z * yy[u].z,
                      t1.y + vv[u].w * yy[u].w};
          if (out_mode == OUT_CHEB) {
            h.x = alpha * (h.x - shift * yy[u].x) + beta * pp[u].x;
            h.y = alpha * (h.y - shift * yy[u].y) + beta * pp[u].y;
            h.z = alpha * (h.z - shift * yy[u].z) + beta * pp[u].z;
            h.w = alpha * (h.w - shift * yy[u].w) + beta * pp[u].w;
          }
          o4[plane_slot4<QX, QY, QZ, CL>(i, crank)] = h;
        }
      }
    }
  }
}

template <int QX, int QY, int QZ, int CL, int NT>
static int launch_shape(const ShapeGroup& g, const FusedArgs& a, const float* X, float* Y, const float* Yprev,
                        const float* V, const double* cheb, int cheb_stride, int out_mode, cudaStream_t st) {
  if (g.qn[0] != QX || g.qn[1] != QY || g.qn[2] != QZ) return 0;
  constexpr int sm = fused_smem_bytes<QX, QY, QZ, CL, NT>();
  FusedArgs b = a;
  b.elems = g.d_elems;
  count_launch();
  if (CL == 1) {
    k_cheb_fused<QX, QY, QZ, CL, NT><<<dim3(g.max_nvec, g.n_elems), NT, sm, st>>>(b, X, Yprev, Y, V, cheb,
                                                                                 cheb_stride, out_mode);
    return 1;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g.max_nvec * CL, g.n_elems);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_cheb_fused<QX, QY, QZ, CL, NT>, b, X, Yprev, Y, V, cheb, cheb_stride, out_mode);
  return 1;
}

// Shared-memory limit (and, for instances with several CTAs per SM, the shared-memory carveout) of every
// fused instance on the current device (per-device attributes: called once per device by context creation
// and by the allocation-free entry point's set-up).
int set_fused_smem_limits() {
  int e = 0;
#define DGDFT_ATTR(a, b, c, cl, nt)                                                                     \
  if (!e) e = allow_max_smem(k_cheb_fused<a, b, c, cl, nt>);                                           \
  if (!e && kFusedThreads / nt > 1)                                                                    \
    e = int(cudaFuncSetAttribute(k_cheb_fused<a, b, c, cl, nt>, cudaFuncAttributePreferredSharedMemoryCarveout, \
                                 100));
  DGDFT_FUSED_SHAPES(DGDFT_ATTR)
#undef DGDFT_ATTR
  return e;
}

// 1 when the fused kernel is instantiated for this Q shape.
int fused_shape_supported(const int qn[3]) {
#define DGDFT_HAS(a, b, c, cl, nt) \
  if (qn[0] == a && qn[1] == b && qn[2] == c) return 1;
  DGDFT_FUSED_SHAPES(DGDFT_HAS)
#undef DGDFT_HAS
  return 0;
}

// Q shapes whose vectors are split over a CTA pair (their lists are split by plane parity)
__device__ __forceinline__ bool split_shape(int qx, int qy, int qz) {
#define DGDFT_SPLIT(a, b, c, cl, nt) \
  if (cl == 2 && qx == a && qy == b && qz == c) return true;
  DGDFT_FUSED_SHAPES(DGDFT_SPLIT)
#undef DGDFT_SPLIT
  return false;
}

// ---- the compact projector-point lists of every fused atom record (once per plan) ----
// One CTA of 256 threads per record: thread t examines the box points 16t .. 16t+15 in (z, y, x) order, a
// block-wide prefix sum (even- and odd-plane counts packed in one word) places the points inside the
// support ball without changing their order; for a shape split over a CTA pair those on even z planes come
// first, indexed in the layout of the planes of their parity.
__global__ void __launch_bounds__(256) k_build_proj_lists(const FusedAtomRec* fat, const double* dtab, int n,
                                                          double inv_rc2, ProjList pl) {
  const int r = blockIdx.x;
  if (r >= n) return;
  const FusedAtomRec at = fat[r];
  __shared__ int scan[256];
  const double* t = dtab + at.dtab;
  const int pitch = 2 * (at.qn[0] / 2 + 1);
  const bool split = split_shape(at.qn[0], at.qn[1], at.qn[2]);
  float gv[16];
  unsigned wv[16];
  int local = 0;   // even-plane count | odd-plane count << 16
#pragma unroll
  for (int q = 0; q < 16; q++) {
    const int e = threadIdx.x * 16 + q;
    const int iz = e >> 8, iy = (e >> 4) & 15, ix = e & 15;
    gv[q] = 0.f;
    wv[q] = 0u;
    if (ix < at.l[0] && iy < at.l[1] && iz < at.l[2]) {
      const double dx = t[ix], dy = t[at.l[0] + iy], dz = t[at.l[0] + at.l[1] + iz];
      const double d2 = dx * dx + dy * dy + dz * dz;
      const double u = 1.0 - d2 * inv_rc2;
      if (u > 0.0) {
        gv[q] = float(exp(-d2 * double(at.inv2s2)) * u * u * u);
        int xx = at.s[0] + ix; if (xx >= at.qn[0]) xx -= at.qn[0];
        int yy = at.s[1] + iy; if (yy >= at.qn[1]) yy -= at.qn[1];
        int zz = at.s[2] + iz; if (zz >= at.qn[2]) zz -= at.qn[2];
        const int upper = split ? (zz & 1) : 0;
        const int zslot = split ? (zz >> 1) : zz;
        wv[q] = unsigned((zslot * at.qn[1] + yy) * pitch + xx) | (unsigned(ix) << 16) |
                (unsigned(iy) << 20) | (unsigned(iz) << 24) | (unsigned(upper) << 31);
        local += upper ? 0x10000 : 1;
      }
    }
  }
  scan[threadIdx.x] = local;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const int v = threadIdx.x >= o ? scan[threadIdx.x - o] : 0;
    __syncthreads();
    scan[threadIdx.x] += v;
    __syncthreads();
  }
  const int total = scan[255];
  const int excl = scan[threadIdx.x] - local;
  int pos_lo = excl & 0xFFFF, pos_hi = (total & 0xFFFF) + (excl >> 16);
  const long long base = (long long)r * kProjCap;
#pragma unroll
  for (int q = 0; q < 16; q++)
    if (gv[q] != 0.f) {
      const int p = (wv[q] >> 31) ? pos_hi++ : pos_lo++;
      pl.gw[base + p] = make_uint2(__float_as_uint(gv[q]), wv[q] & 0x7FFFFFFFu);
    }
  if (threadIdx.x == 255) {
    pl.n[2 * r] = total & 0xFFFF;
    pl.n[2 * r + 1] = total >> 16;
  }
}

void launch_build_proj_lists(const FusedAtomRec* fat, const double* dtab, int n, double r_cut, ProjList pl,
                             cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  k_build_proj_lists<<<n, 256, 0, st>>>(fat, dtab, n, 1.0 / (r_cut * r_cut), pl);
}

// Returns 1 when the fused kernel handled the group (FP32, supported shape, fits shared memory).
int launch_fused_group(const ShapeGroup& g, const HxArgs& h, const float* X, float* Y, const float* Yprev,
                       const float* V, const double* cheb, int cheb_stride, int out_mode, cudaStream_t st) {
  FusedArgs a;
  a.desc = h.desc;
  a.elems = nullptr;
  a.flags = h.flags;
  a.fatoms = h.fatoms;
  a.plist = h.plist;
  a.xo = h.xo;
  a.nvec_mode = h.nvec_mode;
  a.npa = h.n_proj_per_atom;
  int done = 0;
#define DGDFT_LAUNCH(qx, qy, qz, cl, nt) \
  done = done || launch_shape<qx, qy, qz, cl, nt>(g, a, X, Y, Yprev, V, cheb, cheb_stride, out_mode, st);
  DGDFT_FUSED_SHAPES(DGDFT_LAUNCH)
#undef DGDFT_LAUNCH
  return done;
}

}  // namespace dgdft
