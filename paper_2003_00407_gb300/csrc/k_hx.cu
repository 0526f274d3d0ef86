// H x for blocks of vectors on the extended elements (Eq. LocalKS):
//   H x = IFFT( 1/2 |G|^2 FFT(x) ) + V_eff x + sum_{I,l} gamma_{I,l} b_{I,l} <b_{I,l}, x>
// and the fused Chebyshev step  y = alpha (H x - c x) + beta y_prev  (Alg. CheFSI step 2).
//
// Three kernels per application, each batched over (z-plane or column chunk,
// vector, element of one Q shape):
//   plane_forward : load a z-plane, R2C along x (two real rows packed as one
//                   complex row), C2C along y, store the half spectrum;
//                   optionally the projector overlaps <b, x> of the plane;
//   zline         : C2C along z, spectral multiplier, inverse C2C along z;
//   plane_inverse : inverse along y, C2R along x, epilogue (V_eff, nonlocal,
//                   Chebyshev combination) written straight to the output.
#include "fft.cuh"
#include "kernels.h"

namespace dgdft {

constexpr int kMaxPlaneAtoms = 160;

// ---- shape groups run side by side ----
// A batch of several Q shapes (one launch per shape group) runs the groups on kGroupStreams side
// streams forked from and joined back to the caller's stream, so that small groups and the tails of
// large ones overlap instead of queueing.  The groups touch disjoint elements.  One set of streams and
// events per device and host thread, created on first use and kept for the life of the process (no
// destruction at thread or process exit, when the CUDA context may already be gone).
constexpr int kGroupStreams = 4;
struct GroupStreams {
  int dev = -1;
  cudaStream_t s[kGroupStreams];
  cudaEvent_t fork, join[kGroupStreams];
};
static thread_local GroupStreams g_group_streams[16];

template <typename F> static void for_groups(const HxPlan& pl, cudaStream_t st, F&& launch) {
  const int ng = int(pl.groups.size());
  int dev = 0;
  cudaGetDevice(&dev);
  GroupStreams* gs = (ng > 1 && dev >= 0 && dev < 16) ? &g_group_streams[dev] : nullptr;
  if (gs && gs->dev != dev) {
    bool ok = cudaEventCreateWithFlags(&gs->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < kGroupStreams && ok; i++)
      ok = cudaStreamCreateWithFlags(&gs->s[i], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&gs->join[i], cudaEventDisableTiming) == cudaSuccess;
    if (ok) gs->dev = dev;
    else gs = nullptr;   // no side streams: the groups run one after another on st
  }
  if (!gs) {
    for (const ShapeGroup& g : pl.groups) launch(g, st);
    return;
  }
  cudaEventRecord(gs->fork, st);
  const int ns = ng < kGroupStreams ? ng : kGroupStreams;
  for (int i = 0; i < ns; i++) cudaStreamWaitEvent(gs->s[i], gs->fork, 0);
  for (int gi = 0; gi < ng; gi++) launch(pl.groups[gi], gs->s[gi % ns]);
  for (int i = 0; i < ns; i++) {
    cudaEventRecord(gs->join[i], gs->s[i]);
    cudaStreamWaitEvent(st, gs->join[i], 0);
  }
}

int upload_twiddles(const double2* t64, const float2* t32) {
  if (cudaMemcpyToSymbol(g_tw64, t64, sizeof(double2) * kTwiddleCount) != cudaSuccess) return 1;
  if (cudaMemcpyToSymbol(g_tw32, t32, sizeof(float2) * kTwiddleCount) != cudaSuccess) return 1;
  return 0;
}

__host__ int plane_smem_bytes(int qx, int qy, int elem_bytes) {
  const int hx = qx / 2 + 1;
  const int c = 2 * elem_bytes;  // complex
  int r = qy * qx * elem_bytes;                     // real plane
  int c1 = (qy / 2) * qx * c;                       // packed rows
  int c2 = (qy / 2) * qx * c;
  int tmp = (qy / 2) * qx > hx * qy ? (qy / 2) * qx : hx * qy;
  int sp = qy * hx * c;
  return r + c1 + c2 + tmp * c + sp + 16 * 4 * 8 + 1024;  // + projector partials, atom list
}

__host__ int zline_smem_bytes(int qz, int chunk, int elem_bytes) {
  return 2 * qz * chunk * 2 * elem_bytes + 3 * kMaxLine * elem_bytes;
}

// Gaussian-radial projector/well factor g = exp(-d^2 / 2 s^2) (1 - d^2/rc^2)^3 inside rc, else 0
template <typename T> __device__ __forceinline__ T radial_g(T d2, T inv2s2, T inv_rc2) {
  T u = T(1) - d2 * inv_rc2;
  if (u <= T(0)) return T(0);
  return exp(-d2 * inv2s2) * u * u * u;
}

template <typename T>
__global__ void __launch_bounds__(256) k_plane_forward(HxArgs a, const T* __restrict__ X, cplx<T>* __restrict__ S,
                                                       double* __restrict__ P) {
  const int k = a.elems[blockIdx.z];
  const ElemDesc& d = a.desc[k];
  const int v = blockIdx.y, z = blockIdx.x;
  const int nv = a.nvec_mode == 0 ? d.n_blk : (a.nvec_mode == 1 ? d.n_eig : (a.nvec_mode == 2 ? d.n_alb : 1));
  if (v >= nv || z >= d.qn[2]) return;
  if (a.flags && !(a.flags[k] & EF_ACTIVE)) return;
  const int qx = d.qn[0], qy = d.qn[1], hx = qx / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  T* R = reinterpret_cast<T*>(smem);
  cplx<T>* C1 = reinterpret_cast<cplx<T>*>(R + qy * qx);
  cplx<T>* C2 = C1 + (qy / 2) * qx;
  cplx<T>* tmp = C2 + (qy / 2) * qx;
  const int tmpn = (qy / 2) * qx > hx * qy ? (qy / 2) * qx : hx * qy;
  cplx<T>* Sp = tmp + tmpn;

  const T* xp = X + a.xo[k] + (long long)v * d.N + (long long)z * qy * qx;
  for (int i = threadIdx.x; i < qy * qx; i += blockDim.x) R[i] = xp[i];
  __syncthreads();

  if (P != nullptr && d.pa_count > 0 && a.n_proj_per_atom > 0) {
    // projector overlaps of this plane: one warp per atom box, lanes over box points
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const T inv_rc2 = T(1.0 / (a.r_cut * a.r_cut));
    for (int ai = warp; ai < d.pa_count; ai += nw) {
      const AtomBox& b = a.boxes[d.pa_begin + ai];
      int iz = z - b.s[2];
      if (iz < 0) iz += d.qn[2];
      if (iz >= b.l[2]) continue;
      const double* tx = a.dtab + b.toff;
      const double* ty = tx + b.l[0];
      const double* tz = ty + b.l[1];
      const T dz = T(tz[iz]);
      const T inv2s2 = T(0.5 / (b.pwidth * b.pwidth));
      T acc[4] = {T(0), T(0), T(0), T(0)};
      const int npts = b.l[0] * b.l[1];
      for (int p = lane; p < npts; p += 32) {
        const int iy = p / b.l[0], ix = p - iy * b.l[0];
        int yy = b.s[1] + iy; if (yy >= qy) yy -= qy;
        int xx = b.s[0] + ix; if (xx >= qx) xx -= qx;
        const T dx = T(tx[ix]), dy = T(ty[iy]);
        const T d2 = dx * dx + dy * dy + dz * dz;
        const T g = radial_g(d2, inv2s2, inv_rc2);
        const T xv = R[yy * qx + xx] * g;
        acc[0] += xv;
        acc[1] += xv * dx;
        acc[2] += xv * dy;
        acc[3] += xv * dz;
      }
      for (int o = 16; o > 0; o >>= 1)
        for (int l = 0; l < 4; l++) acc[l] += __shfl_xor_sync(0xffffffffu, acc[l], o);
      if (lane == 0) {
        double* pp = P + d.poff + (long long)v * d.n_proj + b.col;
        atomicAdd(pp, double(acc[0]) * b.ns * d.dV);
        if (a.n_proj_per_atom == 4) {
          atomicAdd(pp + 1, double(acc[1]) * b.np * d.dV);
          atomicAdd(pp + 2, double(acc[2]) * b.np * d.dV);
          atomicAdd(pp + 3, double(acc[3]) * b.np * d.dV);
        }
      }
    }
  }

  // pack row pairs (2p, 2p+1) as one complex row
  for (int i = threadIdx.x; i < (qy / 2) * qx; i += blockDim.x) {
    const int p = i / qx, x = i - p * qx;
    C1[i] = cplx<T>{R[(2 * p) * qx + x], R[(2 * p + 1) * qx + x]};
  }
  __syncthreads();
  fft_lines<-1, T>(C1, qx, 1, C2, qx, 1, tmp, qy / 2, d.fx[0], d.fx[1]);
  // unpack: A_k = (Z_k + conj Z_{-k}) / 2,  B_k = (Z_k - conj Z_{-k}) / (2i)
  for (int i = threadIdx.x; i < (qy / 2) * hx; i += blockDim.x) {
    const int p = i / hx, kx = i - p * hx;
    const cplx<T> zk = C2[p * qx + kx];
    const int km = kx == 0 ? 0 : qx - kx;
    const cplx<T> zc = {C2[p * qx + km].re, -C2[p * qx + km].im};
    Sp[(2 * p) * hx + kx] = cplx<T>{T(0.5) * (zk.re + zc.re), T(0.5) * (zk.im + zc.im)};
    Sp[(2 * p + 1) * hx + kx] = cplx<T>{T(0.5) * (zk.im - zc.im), -T(0.5) * (zk.re - zc.re)};
  }
  __syncthreads();
  fft_lines<-1, T>(Sp, 1, hx, Sp, 1, hx, tmp, hx, d.fy[0], d.fy[1]);
  cplx<T>* sp = S + a.so[k] + (long long)v * d.qn[2] * qy * hx + (long long)z * qy * hx;
  for (int i = threadIdx.x; i < qy * hx; i += blockDim.x) sp[i] = Sp[i];
}

template <typename T>
__global__ void __launch_bounds__(256) k_zline(HxArgs a, cplx<T>* __restrict__ S, int mode, int chunk) {
  const int k = a.elems[blockIdx.z];
  const ElemDesc& d = a.desc[k];
  const int v = blockIdx.y;
  const int nv = a.nvec_mode == 0 ? d.n_blk : (a.nvec_mode == 1 ? d.n_eig : (a.nvec_mode == 2 ? d.n_alb : 1));
  const int qx = d.qn[0], qy = d.qn[1], qz = d.qn[2], hx = qx / 2 + 1;
  const int ncol = qy * hx;
  const int c0 = blockIdx.x * chunk;
  if (v >= nv || c0 >= ncol) return;
  if (a.flags && !(a.flags[k] & EF_ACTIVE)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem);
  cplx<T>* tmp = buf + qz * chunk;
  cplx<T>* sp = S + a.so[k] + (long long)v * qz * ncol;
  for (int i = threadIdx.x; i < qz * chunk; i += blockDim.x) {
    const int zz = i / chunk, c = i - zz * chunk;
    buf[i] = (c0 + c < ncol) ? sp[(long long)zz * ncol + c0 + c] : cplx<T>{T(0), T(0)};
  }
  __syncthreads();
  fft_lines<-1, T>(buf, 1, chunk, buf, 1, chunk, tmp, chunk, d.fz[0], d.fz[1]);
  // multiplier tables per axis: kinetic 1/2 G_a^2 / N, or G_a / N for a derivative (Nyquist dropped)
  T* tab = reinterpret_cast<T*>(tmp + qz * chunk);   // [3][kMaxLine]: x, y, z
  const double invN = 1.0 / double(d.N);
  const double twopi = 6.283185307179586476925;
  for (int i = threadIdx.x; i < 3 * kMaxLine; i += blockDim.x) {
    const int ax = i / kMaxLine, kk = i - ax * kMaxLine;
    const int n = ax == 0 ? qx : (ax == 1 ? qy : qz);
    T v = T(0);
    if (kk < n) {
      const int m = kk <= n / 2 ? kk : kk - n;
      const double g = twopi * m / (n * d.h[ax]);
      if (mode == MULT_KINETIC || mode == MULT_TETER) v = T(0.5 * g * g * invN);
      else if (mode == MULT_DX + ax) v = (n % 2 == 0 && kk == n / 2) ? T(0) : T(g * invN);
    }
    tab[i] = v;
  }
  __syncthreads();
  const T sc = T(invN);
  for (int i = threadIdx.x; i < qz * chunk; i += blockDim.x) {
    const int kz = i / chunk, c = i - kz * chunk;
    const int col = c0 + c;
    if (col >= ncol) continue;
    const int ky = col / hx, kx = col - ky * hx;
    cplx<T> s = buf[i];
    if (mode == MULT_KINETIC) {
      s = cscale(s, tab[kx] + tab[kMaxLine + ky] + tab[2 * kMaxLine + kz]);
    } else if (mode == MULT_TETER) {
      // Teter, Payne, Allan (1989): K(x) = (27 + 18x + 12x^2 + 8x^3) / (... + 16x^4), x = (|G|^2/2) / E_v
      const double e = a.mref[(long long)k * a.mref_ld + v];
      const double x = double(tab[kx] + tab[kMaxLine + ky] + tab[2 * kMaxLine + kz]) * double(d.N) / fmax(e, 1e-300);
      const double num = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
      s = cscale(s, T(num / (num + 16.0 * x * x * x * x) * invN));
    } else if (mode == MULT_SCALE) {
      s = cscale(s, sc);
    } else {
      const T f = mode == MULT_DX ? tab[kx] : (mode == MULT_DY ? tab[kMaxLine + ky] : tab[2 * kMaxLine + kz]);
      s = cplx<T>{-s.im * f, s.re * f};
    }
    buf[i] = s;
  }
  __syncthreads();
  fft_lines<1, T>(buf, 1, chunk, buf, 1, chunk, tmp, chunk, d.fz[0], d.fz[1]);
  for (int i = threadIdx.x; i < qz * chunk; i += blockDim.x) {
    const int zz = i / chunk, c = i - zz * chunk;
    if (c0 + c < ncol) sp[(long long)zz * ncol + c0 + c] = buf[i];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_plane_inverse(HxArgs a, const cplx<T>* __restrict__ S, const T* __restrict__ X,
                                                       const T* __restrict__ V, const double* __restrict__ P,
                                                       T* __restrict__ Y, const T* __restrict__ Yprev,
                                                       const double* __restrict__ cheb, int cheb_stride, int out_mode,
                                                       int deriv = -1) {
  const int k = a.elems[blockIdx.z];
  const ElemDesc& d = a.desc[k];
  const int v = blockIdx.y, z = blockIdx.x;
  const int nv = a.nvec_mode == 0 ? d.n_blk : (a.nvec_mode == 1 ? d.n_eig : (a.nvec_mode == 2 ? d.n_alb : 1));
  if (v >= nv || z >= d.qn[2]) return;
  if (a.flags && !(a.flags[k] & EF_ACTIVE)) return;
  const int qx = d.qn[0], qy = d.qn[1], hx = qx / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  T* R = reinterpret_cast<T*>(smem);
  cplx<T>* C1 = reinterpret_cast<cplx<T>*>(R + qy * qx);
  cplx<T>* C2 = C1 + (qy / 2) * qx;
  cplx<T>* tmp = C2 + (qy / 2) * qx;
  const int tmpn = (qy / 2) * qx > hx * qy ? (qy / 2) * qx : hx * qy;
  cplx<T>* Sp = tmp + tmpn;
  int* alist = reinterpret_cast<int*>(Sp + qy * hx);
  __shared__ int na_list;
  __shared__ T acoef[kMaxPlaneAtoms][6];  // gamma_l N_l <b_l, x> for s, px, py, pz; 1/(2 sigma^2)
  const cplx<T>* sp = S + a.so[k] + (long long)v * d.qn[2] * qy * hx + (long long)z * qy * hx;
  if (deriv < 0) {
    for (int i = threadIdx.x; i < qy * hx; i += blockDim.x) Sp[i] = sp[i];
  } else {
    // d/dx or d/dy of a spectrum transformed along x and y only (z still real): i G_a / (qx qy) (Nyquist
    // dropped), the same as the z-line pass with the derivative multiplier, whose z transforms cancel
    const int n = deriv == 0 ? qx : qy;
    const double f = 6.283185307179586476925 / (n * d.h[deriv]) / (double(qx) * double(qy));
    for (int i = threadIdx.x; i < qy * hx; i += blockDim.x) {
      const int kk = deriv == 0 ? i % hx : i / hx;
      const int m = kk <= n / 2 ? kk : kk - n;
      const T g = (n % 2 == 0 && kk == n / 2) ? T(0) : T(f * m);
      const cplx<T> s = sp[i];
      Sp[i] = cplx<T>{-s.im * g, s.re * g};
    }
  }
  if (threadIdx.x == 0) {
    // atom boxes that meet this plane (for the nonlocal term)
    int n = 0;
    if (out_mode != OUT_RAW && P != nullptr && a.n_proj_per_atom > 0) {
      const double* pv0 = P + d.poff + (long long)v * d.n_proj;
      for (int ai = 0; ai < d.pa_count && n < kMaxPlaneAtoms; ai++) {
        const AtomBox& b = a.boxes[d.pa_begin + ai];
        int iz = z - b.s[2];
        if (iz < 0) iz += d.qn[2];
        if (iz < b.l[2]) {
          alist[n] = ai;
          acoef[n][0] = T(b.gamma[0] * b.ns * pv0[b.col]);
          for (int l = 1; l < 4; l++)
            acoef[n][l] = a.n_proj_per_atom == 4 ? T(b.gamma[l] * b.np * pv0[b.col + l]) : T(0);
          acoef[n][4] = T(0.5 / (b.pwidth * b.pwidth));
          acoef[n][5] = T(b.l[0] + b.l[1] + iz);   // dtab index of this plane's z displacement (relative)
          n++;
        }
      }
    }
    na_list = n;
  }
  __syncthreads();
  fft_lines<1, T>(Sp, 1, hx, Sp, 1, hx, tmp, hx, d.fy[0], d.fy[1]);
  // rebuild the full complex rows Z = A + i B from the two half spectra
  for (int i = threadIdx.x; i < (qy / 2) * qx; i += blockDim.x) {
    const int p = i / qx, kk = i - p * qx;
    cplx<T> A, B;
    if (kk < hx) {
      A = Sp[(2 * p) * hx + kk];
      B = Sp[(2 * p + 1) * hx + kk];
      C1[i] = cplx<T>{A.re - B.im, A.im + B.re};
    } else {
      A = Sp[(2 * p) * hx + (qx - kk)];
      B = Sp[(2 * p + 1) * hx + (qx - kk)];
      C1[i] = cplx<T>{A.re + B.im, -A.im + B.re};
    }
  }
  __syncthreads();
  fft_lines<1, T>(C1, qx, 1, C2, qx, 1, tmp, qy / 2, d.fx[0], d.fx[1]);

  const long long base = a.xo[k] + (long long)v * d.N + (long long)z * qy * qx;
  if (out_mode == OUT_RAW) {
    for (int i = threadIdx.x; i < qy * qx; i += blockDim.x) {
      const int y = i / qx, x = i - y * qx;
      const cplx<T> c = C2[(y >> 1) * qx + x];
      Y[base + i] = (y & 1) ? c.im : c.re;
    }
    return;
  }
  double alpha = 1.0, shift = 0.0, beta = 0.0;
  if (out_mode == OUT_CHEB) {
    alpha = cheb[k * cheb_stride + 0];
    shift = cheb[k * cheb_stride + 1];
    beta = cheb[k * cheb_stride + 2];
  }
  const T* vq = V + d.voff + (long long)z * qy * qx;
  const T inv_rc2 = T(1.0 / (a.r_cut * a.r_cut));
  const int nal = na_list;
  for (int i = threadIdx.x; i < qy * qx; i += blockDim.x) {
    const int y = i / qx, x = i - y * qx;
    const cplx<T> c = C2[(y >> 1) * qx + x];
    const T tx = (y & 1) ? c.im : c.re;
    const T xv = X[base + i];
    T hxv = tx + vq[i] * xv;
    for (int li = 0; li < nal; li++) {
      const AtomBox& b = a.boxes[d.pa_begin + alist[li]];
      int iy = y - b.s[1]; if (iy < 0) iy += qy;
      if (iy >= b.l[1]) continue;
      int ix = x - b.s[0]; if (ix < 0) ix += qx;
      if (ix >= b.l[0]) continue;
      const double* tx0 = a.dtab + b.toff;
      const T* ac = acoef[li];
      const T dx = T(tx0[ix]), dy = T(tx0[b.l[0] + iy]), dz = T(tx0[int(ac[5])]);
      const T g = radial_g(dx * dx + dy * dy + dz * dz, ac[4], inv_rc2);
      if (g == T(0)) continue;
      hxv += g * (ac[0] + ac[1] * dx + ac[2] * dy + ac[3] * dz);
    }
    T out;
    if (out_mode == OUT_CHEB) {
      out = T(alpha) * (hxv - T(shift) * xv);
      if (Yprev != nullptr && beta != 0.0) out += T(beta) * Yprev[base + i];
    } else {
      out = hxv;
    }
    Y[base + i] = out;
  }
}

// ---------------------------------------------------------------------------
template <typename T>
void launch_hx(const HxPlan& pl, const HxArgs& args, const T* X, T* Y, const T* Yprev, const T* V, cplx<T>* S,
               double* P, const double* cheb, int cheb_stride, int out_mode, int mult_mode, cudaStream_t st) {
  for_groups(pl, st, [&](const ShapeGroup& g, cudaStream_t st) {
    HxArgs a = args;
    a.elems = g.d_elems;
    if constexpr (sizeof(T) == 4) {
      if (mult_mode == MULT_KINETIC && out_mode != OUT_RAW && g.fused_ok &&
          launch_fused_group(g, a, X, Y, Yprev, V, cheb, cheb_stride, out_mode, st))
        return;
    }
    const int eb = sizeof(T);
    const int smA = plane_smem_bytes(g.qn[0], g.qn[1], eb);
    const int chunk = g.zchunk;
    const int smB = zline_smem_bytes(g.qn[2], chunk, eb);
    const int hx = g.qn[0] / 2 + 1;
    dim3 gA(g.qn[2], g.max_nvec, g.n_elems);
    dim3 gB((g.qn[1] * hx + chunk - 1) / chunk, g.max_nvec, g.n_elems);
    count_launch(); k_plane_forward<T><<<gA, 256, smA, st>>>(a, X, S, (out_mode == OUT_RAW) ? nullptr : P);
    count_launch(); k_zline<T><<<gB, 256, smB, st>>>(a, S, mult_mode, chunk);
    count_launch(); k_plane_inverse<T><<<gA, 256, smA, st>>>(a, S, X, V, (out_mode == OUT_RAW) ? nullptr : P, Y, Yprev, cheb,
                                              cheb_stride, out_mode);
  });
}

// forward transform only (used by the DG gradients): spectrum of X in S
template <typename T>
void launch_forward(const HxPlan& pl, const HxArgs& args, const T* X, cplx<T>* S, cudaStream_t st) {
  for_groups(pl, st, [&](const ShapeGroup& g, cudaStream_t st) {
    HxArgs a = args;
    a.elems = g.d_elems;
    dim3 gA(g.qn[2], g.max_nvec, g.n_elems);
    count_launch(); k_plane_forward<T><<<gA, 256, plane_smem_bytes(g.qn[0], g.qn[1], sizeof(T)), st>>>(a, X, S, nullptr);
  });
}

template <typename T>
void launch_zline(const HxPlan& pl, const HxArgs& args, cplx<T>* S, int mult_mode, cudaStream_t st) {
  for_groups(pl, st, [&](const ShapeGroup& g, cudaStream_t st) {
    HxArgs a = args;
    a.elems = g.d_elems;
    const int hx = g.qn[0] / 2 + 1;
    dim3 gB((g.qn[1] * hx + g.zchunk - 1) / g.zchunk, g.max_nvec, g.n_elems);
    count_launch(); k_zline<T><<<gB, 256, zline_smem_bytes(g.qn[2], g.zchunk, sizeof(T)), st>>>(a, S, mult_mode, g.zchunk);
  });
}

template <typename T>
void launch_inverse_raw(const HxPlan& pl, const HxArgs& args, const cplx<T>* S, T* Y, cudaStream_t st, int deriv) {
  for_groups(pl, st, [&](const ShapeGroup& g, cudaStream_t st) {
    HxArgs a = args;
    a.elems = g.d_elems;
    dim3 gA(g.qn[2], g.max_nvec, g.n_elems);
    count_launch(); k_plane_inverse<T><<<gA, 256, plane_smem_bytes(g.qn[0], g.qn[1], sizeof(T)), st>>>(
        a, S, nullptr, nullptr, nullptr, Y, nullptr, nullptr, 0, OUT_RAW, deriv);
  });
}

int set_hx_smem_limits() {
  int e = 0;
  e |= allow_max_smem(k_plane_forward<float>);
  e |= allow_max_smem(k_plane_forward<double>);
  e |= allow_max_smem(k_plane_inverse<float>);
  e |= allow_max_smem(k_plane_inverse<double>);
  e |= allow_max_smem(k_zline<float>);
  e |= allow_max_smem(k_zline<double>);
  return e;
}

template void launch_hx<float>(const HxPlan&, const HxArgs&, const float*, float*, const float*, const float*,
                               cplx<float>*, double*, const double*, int, int, int, cudaStream_t);
template void launch_hx<double>(const HxPlan&, const HxArgs&, const double*, double*, const double*, const double*,
                                cplx<double>*, double*, const double*, int, int, int, cudaStream_t);
template void launch_forward<double>(const HxPlan&, const HxArgs&, const double*, cplx<double>*, cudaStream_t);
template void launch_zline<double>(const HxPlan&, const HxArgs&, cplx<double>*, int, cudaStream_t);
template void launch_inverse_raw<double>(const HxPlan&, const HxArgs&, const cplx<double>*, double*, cudaStream_t, int);

}  // namespace dgdft
