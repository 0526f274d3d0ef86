// Fused FP32 Chebyshev step for one vector per CTA (Eq. LocalKS, Alg. CheFSI step 2):
//   y_out = alpha (H y - c y) + beta y_prev      (or y_out = H y)
// with H y = IFFT(1/2 |G|^2 FFT(y)) + V y + sum_{I,l} gamma b <b, y>.
// The half spectrum [QZ][QY][QX/2+1] of the vector stays in shared memory for the
// whole step, so the vector is read once from HBM (plus an L2 re-read in the
// epilogue), y_prev is read once and y_out written once.
// Phases (one __syncthreads between each):
//   1 x-rows: load, projector overlaps <b, y>, R2C along x (length QX via a
//     complex transform of QX/2), store the row's half spectrum;
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

// Length-N transform split over a lane pair (lanes i and i+16, h = lane >> 4, so that a
// half-warp holds 16 consecutive lines: conflict-free shared accesses); each lane holds N/2 points.
// Forward (radix-2 decimation in time): lane h loads x[2m + h], computes the half
// transform, the odd lane twiddles by w_N^k, one exchange gives lane h the outputs
// X[k + h N/2] (X_k = E_k + w^k O_k, X_{k+N/2} = E_k - w^k O_k).
template <int N> __device__ __forceinline__ void pair_fft_fwd(cf (&x)[N / 2], int h) {
  reg_fft<N / 2, -1>(x);
  const float s = h ? -1.f : 1.f;
#pragma unroll
  for (int k = 0; k < N / 2; k++) {
    const cf w = twc<N, -1>(k);
    const cf mine = h ? cmul(x[k], w) : x[k];
    const cf recv = {__shfl_xor_sync(0xffffffffu, mine.re, 16), __shfl_xor_sync(0xffffffffu, mine.im, 16)};
    x[k] = cf{fmaf(s, mine.re, recv.re), fmaf(s, mine.im, recv.im)};
  }
}
// Inverse (radix-2 decimation in frequency), unnormalised: lane h holds X[k + h N/2] on
// entry and x[2m + h] on exit (A_k = X_k + X_{k+N/2}, B_k = (X_k - X_{k+N/2}) w^{-k}).
template <int N> __device__ __forceinline__ void pair_fft_inv(cf (&x)[N / 2], int h) {
  const float s = h ? -1.f : 1.f;
#pragma unroll
  for (int k = 0; k < N / 2; k++) {
    const cf mine = x[k];
    const cf recv = {__shfl_xor_sync(0xffffffffu, mine.re, 16), __shfl_xor_sync(0xffffffffu, mine.im, 16)};
    const cf t = {fmaf(s, mine.re, recv.re), fmaf(s, mine.im, recv.im)};
    x[k] = h ? cmul(t, twc<N, 1>(k)) : t;
  }
  reg_fft<N / 2, 1>(x);
}

struct FusedArgs {
  const ElemDesc* desc;
  const int* elems;
  const int* flags;
  const FusedAtomRec* fatoms;
  const float* dtab32;
  const float* gtab;
  const long long* xo;
  int nvec_mode;
  int npa;
  float inv_rc2;
};

// g(d) = exp(-d^2 / 2 sigma^2) (1 - d^2/rc^2)^3 inside r_cut (else 0) at every point of a Q box,
// stored [atom][iz][iy][ix] in a 16^3 block per atom (the element's 80 vectors and all filter
// steps share it).
__global__ void k_build_gtab(BatchArgs b, const FusedAtomRec* fatoms, const float* dtab32, float inv_rc2,
                             float* gtab) {
  const int k = blockIdx.z, ai = blockIdx.y;
  const ElemDesc& d = b.desc[k];
  if (ai >= d.pa_count) return;
  const FusedAtomRec& at = fatoms[d.pa_begin + ai];
  const float* tx = dtab32 + d.tab_off + at.toff;
  float* out = gtab + d.gtab_off + (long long)ai * 4096;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 4096; i += gridDim.x * blockDim.x) {
    const int ix = i & 15, iy = (i >> 4) & 15, iz = i >> 8;
    float g = 0.f;
    if (ix < at.l[0] && iy < at.l[1] && iz < at.l[2]) {
      const float dx = tx[ix], dy = tx[at.l[0] + iy], dz = tx[at.l[0] + at.l[1] + iz];
      const float d2 = dx * dx + dy * dy + dz * dz;
      const float u = 1.f - d2 * inv_rc2;
      if (u > 0.f) g = expf(-d2 * at.inv2s2) * u * u * u;
    }
    out[i] = g;
  }
}

void launch_build_gtab(const BatchArgs& b, const FusedAtomRec* fatoms, const float* dtab32, float r_cut, int max_pa,
                       float* gtab, cudaStream_t st) {
  if (max_pa <= 0) return;
  count_launch(); k_build_gtab<<<dim3(4, max_pa, b.M), 256, 0, st>>>(b, fatoms, dtab32, 1.f / (r_cut * r_cut), gtab);
}

constexpr int kFusedThreads = 544;   // 17 warps: y tasks (2 x 17 x 48) = 3 rounds, z tasks (2 x 17 x 32) = 2 rounds
constexpr int kFusedWarps = kFusedThreads / 32;
constexpr int kFusedMaxAtoms = 96;
constexpr int kFusedMaxTab = 3072;   // floats of displacement tables (+ 32 x-factors per atom) per CTA

template <int QX, int QY, int QZ> constexpr int fused_smem_bytes() {
  return (QX / 2 + 1) * QY * QZ * 8 + kFusedMaxTab * 4;
}

// Nonlocal work item: one z-slice iz of one atom's box, done by one warp.  The
// slice's x-rows are walked two at a time (lanes 0-15 row A, 16-31 row B; an
// x-row of a box has at most 16 points), only over the rows whose |dy| can be
// inside r_cut.  PROJ accumulates the overlap sums (s, x, y, z components
// without the norms) of the real rows in buf into acc; otherwise the nonlocal
// term g (c_s + c_x dx + c_y dy + c_z dz) is added into buf.
// Nonlocal work item: two z-slices (iz = 2 zq + lane/16) of one atom's box; each
// lane owns one x-row (iy = lane % 16) and its 16 points.  The row's radial
// factors g come from the element's table (four 128-bit loads, 0 outside the
// sphere and the box).  PROJ accumulates the overlap sums (s, x, y, z
// components without the norms) of the real rows in buf into acc; otherwise the
// nonlocal term g (c_s + c_x dx + c_y dy + c_z dz) is added into buf.
struct GRow {
  float4 q[4];
};

// the 16 radial factors of this lane's x-row of item (atom ai, z-slice pair zq)
__device__ __forceinline__ GRow load_grow(const float* __restrict__ gatom, int zq) {
  const int lane = threadIdx.x & 31;
  const int iy = lane & 15, iz = 2 * zq + (lane >> 4);
  GRow r;
  if (iz < 16) {
    const float4* g4 = reinterpret_cast<const float4*>(gatom + (iz * 16 + iy) * 16);
    r.q[0] = __ldg(g4); r.q[1] = __ldg(g4 + 1); r.q[2] = __ldg(g4 + 2); r.q[3] = __ldg(g4 + 3);
  } else {
    r.q[0] = r.q[1] = r.q[2] = r.q[3] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  return r;
}

// Application from the element's radial-factor table (16 factors of this lane's row, loaded as four
// 128-bit words; zero outside the sphere and the box): buf += g (b0 + b1 i).
template <int QX, int QY, int QZ>
__device__ __forceinline__ void atom_rows16_apply(const FusedAtomRec& at, const float* __restrict__ gatom, int zq,
                                                  const float* tabs, float hx, float* buf, int pitch,
                                                  const float* coef) {
  const int lane = threadIdx.x & 31;
  const int iy = lane & 15, iz = 2 * zq + (lane >> 4);
  if (!(iy < at.l[1] && iz < at.l[2])) return;
  const float* tx = tabs + at.toff;
  const float dx0 = tx[0];
  const float dy = tx[at.l[0] + iy], dz = tx[at.l[0] + at.l[1] + iz];
  const float4* g4 = reinterpret_cast<const float4*>(gatom + (iz * 16 + iy) * 16);
  const float4 q0 = __ldg(g4), q1 = __ldg(g4 + 1), q2 = __ldg(g4 + 2), q3 = __ldg(g4 + 3);
  const float g[16] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w, q3.x, q3.y, q3.z, q3.w};
  int yy = at.s[1] + iy;
  if (yy >= QY) yy -= QY;
  int zz = at.s[2] + iz;
  if (zz >= QZ) zz -= QZ;
  float* rbuf = buf + (zz * QY + yy) * pitch;
  const float b0 = coef[0] + coef[2] * dy + coef[3] * dz + coef[1] * dx0;
  const float b1 = coef[1] * hx;
  const bool nowrap = at.s[0] + 16 <= QX;
#pragma unroll
  for (int i = 0; i < 16; i++) {
    int xx = at.s[0] + i;
    if (!nowrap && xx >= QX) xx -= QX;
    if (g[i] != 0.f) atomicAdd(rbuf + xx, g[i] * fmaf(b1, float(i), b0));
  }
}

// xf: per-atom x factors in shared memory: xf[i] = exp(-dx_i^2 / 2 sigma^2) and xf[16 + i] = dx_i^2 / rc^2
// (0 and 1e30 for i beyond the box), so g = e_row xf[i] max(0, rem_row - xf[16 + i])^3.
template <int QX, int QY, int QZ, bool PROJ>
__device__ __forceinline__ void atom_rows16(const FusedAtomRec& at, const float* xf, int zq, const float* tabs,
                                            float hx, float inv_rc2, float* buf, int pitch, const float* coef,
                                            float acc[4]) {
  const int lane = threadIdx.x & 31;
  const int iy = lane & 15, iz = 2 * zq + (lane >> 4);
  const float* tx = tabs + at.toff;
  float s = 0.f, si = 0.f;
  float dy = 0.f, dz = 0.f;
  const float dx0 = tx[0];   // box displacements are affine: dx_i = dx0 + i hx
  bool row_ok = iy < at.l[1] && iz < at.l[2];
  if (row_ok) {
    dy = tx[at.l[0] + iy];
    dz = tx[at.l[0] + at.l[1] + iz];
  }
  const float dyz2 = dy * dy + dz * dz;
  const float rem = 1.f - dyz2 * inv_rc2;
  row_ok = row_ok && rem > 0.f;
  if (row_ok) {
    const float erow = __expf(-dyz2 * at.inv2s2);
    int yy = at.s[1] + iy;
    if (yy >= QY) yy -= QY;
    int zz = at.s[2] + iz;
    if (zz >= QZ) zz -= QZ;
    float* rbuf = buf + (zz * QY + yy) * pitch;
    // nonlocal term g (c_s + c_x dx + c_y dy + c_z dz) = g (b0 + b1 i)
    const float b0 = PROJ ? 0.f : erow * (coef[0] + coef[2] * dy + coef[3] * dz + coef[1] * dx0);
    const float b1 = PROJ ? 0.f : erow * coef[1] * hx;
    const bool nowrap = at.s[0] + 16 <= QX;
#pragma unroll
    for (int i = 0; i < 16; i++) {
      int xx = at.s[0] + i;
      if (!nowrap && xx >= QX) xx -= QX;
      const float u = fmaxf(rem - xf[16 + i], 0.f);
      const float g = xf[i] * u * u * u;
      if (PROJ) {
        const float gy = g * rbuf[xx];
        s += gy;
        si = fmaf(gy, float(i), si);
      } else if (g != 0.f) {
        atomicAdd(rbuf + xx, g * fmaf(b1, float(i), b0));
      }
    }
    if (PROJ) { s *= erow; si *= erow; }
  }
  if (PROJ) {
    float sx = fmaf(dx0, s, hx * si), sy = s * dy, sz = s * dz;   // sum g y dx = dx0 s + hx sum i g y
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, o);
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    acc[0] = s; acc[1] = sx; acc[2] = sy; acc[3] = sz;
  }
}

template <int QX, int QY, int QZ>
__global__ void __launch_bounds__(kFusedThreads, 1)
    k_cheb_fused(FusedArgs a, const float* __restrict__ Y, const float* __restrict__ Yprev, float* __restrict__ Yout,
                 const float* __restrict__ V, const double* __restrict__ cheb, int cheb_stride, int out_mode) {
  constexpr int HX = QX / 2 + 1;
  constexpr int PITCH = 2 * HX;            // floats per x-row slot (real row or its half spectrum)
  constexpr int NROW = QY * QZ;
  constexpr int NF4 = NROW * QX / 4;       // float4 of the vector
  const int k = a.elems[blockIdx.y];
  const int v = blockIdx.x;
  const ElemDesc& d = a.desc[k];
  const int nv = a.nvec_mode == 0 ? d.n_blk : (a.nvec_mode == 1 ? d.n_eig : (a.nvec_mode == 2 ? d.n_alb : 1));
  if (v >= nv) return;
  if (a.flags && !(a.flags[k] & EF_ACTIVE)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  cf* S = reinterpret_cast<cf*>(smem);                               // [QZ][QY][HX]
  float* Sf = reinterpret_cast<float*>(smem);
  float* tabs = reinterpret_cast<float*>(smem + HX * QY * QZ * 8);   // displacement tables
  __shared__ FusedAtomRec atoms[kFusedMaxAtoms];
  __shared__ float pacc[kFusedMaxAtoms][4];
  __shared__ float kmul[3][kMaxLine];
  __shared__ int item_off[kFusedMaxAtoms + 1];   // nonlocal work items (atom, z-slice pair), atom-major
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int na = a.npa > 0 ? d.pa_count : 0;

  // ---- prologue: atom records and tables (cooperative copies), multiplier tables ----
  {
    const int* src = reinterpret_cast<const int*>(a.fatoms + d.pa_begin);
    int* dst = reinterpret_cast<int*>(atoms);
    constexpr int W = sizeof(FusedAtomRec) / 4;
    for (int i = threadIdx.x; i < na * W; i += blockDim.x) dst[i] = __ldg(src + i);
    if (na > 0)
      for (int i = threadIdx.x; i < d.tab_len; i += blockDim.x) tabs[i] = __ldg(a.dtab32 + d.tab_off + i);
    for (int i = threadIdx.x; i < 3 * kMaxLine; i += blockDim.x) {
      const int ax = i / kMaxLine, kk = i % kMaxLine;
      const int n = ax == 0 ? QX : (ax == 1 ? QY : QZ);
      const int m = kk <= n / 2 ? kk : kk - n;
      kmul[ax][kk] = kk < n ? d.kscale[ax] * float(m * m) : 0.f;
    }
    for (int i = threadIdx.x; i < kFusedMaxAtoms * 4; i += blockDim.x) (&pacc[0][0])[i] = 0.f;
  }
  __syncthreads();
  float* xfac = tabs + d.tab_len;   // [na][32]
  for (int i = threadIdx.x; i < na * 32; i += blockDim.x) {
    const int ai = i >> 5, j = i & 31, ix = j & 15;
    const FusedAtomRec& at = atoms[ai];
    const float dx = tabs[at.toff] + float(ix) * float(d.h[0]);
    const bool in = ix < at.l[0];
    xfac[i] = j < 16 ? (in ? __expf(-dx * dx * at.inv2s2) : 0.f) : (in ? dx * dx * a.inv_rc2 : 1e30f);
  }
  if (threadIdx.x == 0) {
    item_off[0] = 0;
    for (int ai = 0; ai < na; ai++) item_off[ai + 1] = item_off[ai] + (atoms[ai].l[2] + 1) / 2;
  }
  const float inv_rc2 = a.inv_rc2;
  const float hy = float(d.h[1]);
  const float hx = float(d.h[0]);
  const long long vbase = a.xo[k] + (long long)v * (QX * QY * QZ);
  const float4* y4 = reinterpret_cast<const float4*>(Y + vbase);

  // ---- phase 1a: the real vector into the row slots (coalesced float4 loads) ----
#pragma unroll 4
  for (int i = threadIdx.x; i < NF4; i += kFusedThreads) {
    const int r = i / (QX / 4), c = i % (QX / 4);
    const float4 q = __ldg(y4 + i);
    float2* dst = reinterpret_cast<float2*>(Sf + r * PITCH + 4 * c);
    dst[0] = make_float2(q.x, q.y);
    dst[1] = make_float2(q.z, q.w);
  }
  __syncthreads();
  const int n_items = item_off[na];
  // ---- phase 1b: projector overlaps <b, y> from the real rows ----
  {
    int ai = 0;
    for (int it = warp; it < n_items; it += kFusedWarps) {
      while (item_off[ai + 1] <= it) ai++;
      float acc[4];
      atom_rows16<QX, QY, QZ, true>(atoms[ai], xfac + ai * 32, it - item_off[ai], tabs, hx, inv_rc2, Sf, PITCH,
                                    nullptr, acc);
      if (lane < 4) atomicAdd(&pacc[ai][lane], lane == 0 ? acc[0] : lane == 1 ? acc[1] : lane == 2 ? acc[2] : acc[3]);
    }
  }
  __syncthreads();
  // ---- phase 1c: R2C along x in each row slot: z = x_even + i x_odd, X_k = E_k + w^k O_k ----
  for (int r = threadIdx.x; r < NROW; r += blockDim.x) {
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
  for (int l0 = 0; l0 < HX * QZ; l0 += 16 * kFusedWarps) {
    const int h = lane >> 4, lt = l0 + warp * 16 + (lane & 15);
    const bool ok = lt < HX * QZ;
    const int l = ok ? lt : 0;
    const int kx = l % HX, z = l / HX;
    cf* base = S + (long long)z * QY * HX + kx;
    cf q[QY / 2];
#pragma unroll
    for (int m = 0; m < QY / 2; m++) q[m] = ok ? base[(2 * m + h) * HX] : cf{0.f, 0.f};
    pair_fft_fwd<QY>(q, h);
    if (ok) {
#pragma unroll
      for (int m = 0; m < QY / 2; m++) base[(m + h * (QY / 2)) * HX] = q[m];
    }
  }
  if (threadIdx.x < na) {
    // c_l = gamma_l N_l^2 dV <...>: the term at a point is g (c_s + c_x dx + c_y dy + c_z dz)
    float* pa = pacc[threadIdx.x];
    const float* c = atoms[threadIdx.x].c;
    pa[0] *= c[0]; pa[1] *= c[1]; pa[2] *= c[2]; pa[3] *= c[3];
  }
  __syncthreads();
  // ---- phase 3: z lines (lane pairs): forward, 1/2|G|^2 / N, inverse ----
  for (int l0 = 0; l0 < HX * QY; l0 += 16 * kFusedWarps) {
    const int h = lane >> 4, lt = l0 + warp * 16 + (lane & 15);
    const bool ok = lt < HX * QY;
    const int l = ok ? lt : 0;
    const int kx = l % HX, ky = l / HX;
    cf* base = S + l;
    cf q[QZ / 2];
#pragma unroll
    for (int m = 0; m < QZ / 2; m++) q[m] = ok ? base[(long long)(2 * m + h) * QY * HX] : cf{0.f, 0.f};
    pair_fft_fwd<QZ>(q, h);
    const float kxy = kmul[0][kx] + kmul[1][ky];
#pragma unroll
    for (int m = 0; m < QZ / 2; m++) q[m] = cscale(q[m], kxy + kmul[2][m + h * (QZ / 2)]);
    pair_fft_inv<QZ>(q, h);
    if (ok) {
#pragma unroll
      for (int m = 0; m < QZ / 2; m++) base[(long long)(2 * m + h) * QY * HX] = q[m];
    }
  }
  __syncthreads();
  // ---- phase 4: y lines inverse (lane pairs) ----
  for (int l0 = 0; l0 < HX * QZ; l0 += 16 * kFusedWarps) {
    const int h = lane >> 4, lt = l0 + warp * 16 + (lane & 15);
    const bool ok = lt < HX * QZ;
    const int l = ok ? lt : 0;
    const int kx = l % HX, z = l / HX;
    cf* base = S + (long long)z * QY * HX + kx;
    cf q[QY / 2];
#pragma unroll
    for (int m = 0; m < QY / 2; m++) q[m] = ok ? base[(m + h * (QY / 2)) * HX] : cf{0.f, 0.f};
    pair_fft_inv<QY>(q, h);
    if (ok) {
#pragma unroll
      for (int m = 0; m < QY / 2; m++) base[(2 * m + h) * HX] = q[m];
    }
  }
  __syncthreads();
  // ---- phase 5a: C2R along x; each row slot then holds T y (real) ----
  for (int r = threadIdx.x; r < NROW; r += blockDim.x) {
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
  // ---- phase 5b: nonlocal application ((atom, z-slice pair) items, shared atomics) ----
  {
    int ai = 0;
    for (int it = warp; it < n_items; it += kFusedWarps) {
      while (item_off[ai + 1] <= it) ai++;
      atom_rows16_apply<QX, QY, QZ>(atoms[ai], a.gtab + d.gtab_off + (long long)ai * 4096, it - item_off[ai], tabs,
                                    hx, Sf, PITCH, pacc[ai]);
    }
  }
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
#pragma unroll 4
  for (int i = threadIdx.x; i < NF4; i += kFusedThreads) {
    const int r = i / (QX / 4), c = i % (QX / 4);
    const float2* tr = reinterpret_cast<const float2*>(Sf + r * PITCH + 4 * c);
    const float2 t0 = tr[0], t1 = tr[1];
    const float4 yy = __ldg(y4 + i), vv = __ldg(v4 + i);
    float4 h = {t0.x + vv.x * yy.x, t0.y + vv.y * yy.y, t1.x + vv.z * yy.z, t1.y + vv.w * yy.w};
    if (out_mode == OUT_CHEB) {
      h.x = alpha * (h.x - shift * yy.x);
      h.y = alpha * (h.y - shift * yy.y);
      h.z = alpha * (h.z - shift * yy.z);
      h.w = alpha * (h.w - shift * yy.w);
      if (p4 != nullptr) {
        const float4 pp = __ldg(p4 + i);
        h.x += beta * pp.x; h.y += beta * pp.y; h.z += beta * pp.z; h.w += beta * pp.w;
      }
    }
    o4[i] = h;
  }
}

template <int QX, int QY, int QZ>
static int launch_shape(const ShapeGroup& g, const FusedArgs& a, const float* X, float* Y, const float* Yprev,
                        const float* V, const double* cheb, int cheb_stride, int out_mode, cudaStream_t st) {
  if (g.qn[0] != QX || g.qn[1] != QY || g.qn[2] != QZ) return 0;
  static bool attr = false;
  constexpr int sm = fused_smem_bytes<QX, QY, QZ>();
  if (!attr) {
    if (allow_max_smem(k_cheb_fused<QX, QY, QZ>)) return 0;
    attr = true;
  }
  FusedArgs b = a;
  b.elems = g.d_elems;
  dim3 grid(g.max_nvec, g.n_elems);
  count_launch(); k_cheb_fused<QX, QY, QZ><<<grid, kFusedThreads, sm, st>>>(b, X, Yprev, Y, V, cheb, cheb_stride, out_mode);
  return 1;
}

// 1 when the fused kernel is instantiated for this Q shape.
int fused_shape_supported(const int qn[3]) {
  static const int shapes[][3] = {{32, 32, 48}, {16, 16, 16}, {32, 32, 32}, {24, 24, 32}, {24, 24, 48}};
  for (const auto& s : shapes)
    if (qn[0] == s[0] && qn[1] == s[1] && qn[2] == s[2]) return 1;
  return 0;
}

// Returns 1 when the fused kernel handled the group (FP32, supported shape, fits shared memory).
int launch_fused_group(const ShapeGroup& g, const HxArgs& h, const float* X, float* Y, const float* Yprev,
                       const float* V, const double* cheb, int cheb_stride, int out_mode, cudaStream_t st) {
  FusedArgs a;
  a.desc = h.desc;
  a.elems = nullptr;
  a.flags = h.flags;
  a.fatoms = h.fatoms;
  a.dtab32 = h.dtab32;
  a.gtab = h.gtab;
  a.xo = h.xo;
  a.nvec_mode = h.nvec_mode;
  a.npa = h.n_proj_per_atom;
  a.inv_rc2 = float(1.0 / (h.r_cut * h.r_cut));
  int done = 0;
  done = done || launch_shape<32, 32, 48>(g, a, X, Y, Yprev, V, cheb, cheb_stride, out_mode, st);
  done = done || launch_shape<16, 16, 16>(g, a, X, Y, Yprev, V, cheb, cheb_stride, out_mode, st);
  done = done || launch_shape<32, 32, 32>(g, a, X, Y, Yprev, V, cheb, cheb_stride, out_mode, st);
  done = done || launch_shape<24, 24, 32>(g, a, X, Y, Yprev, V, cheb, cheb_stride, out_mode, st);
  done = done || launch_shape<24, 24, 48>(g, a, X, Y, Yprev, V, cheb, cheb_stride, out_mode, st);
  return done;
}

}  // namespace dgdft
