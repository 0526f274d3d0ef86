// dgdft_apply_hamiltonian_noalloc: the FP32 Hamiltonian application without any
// device allocation.  For callers that cannot call cudaMalloc/cudaFree: hosts
// whose device memory is entirely reserved by another allocator (frameworks
// that pre-reserve most of HBM for their own pool), and latency-critical
// callers that cannot accept the device-wide synchronisation that
// cudaMalloc/cudaFree imply.  Every scratch table lives in the file-scope
// device array below; inputs and outputs are the caller's.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dgdft.h"
#include "kernels.h"
#include "plan.h"

namespace dgdft {

int fail(dgdft_ctx* c, int code, const std::string& msg);

// Scratch of the allocation-free entry point.  Every GPU that loads the library
// holds these 24 MiB until the process exits.  All calls share it and it keeps
// the contents of the last call: calls that overlap on the GPU (other streams,
// other host threads) race on it.
constexpr size_t kNoAllocScratchBytes = size_t(24) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
  bool ready;
  unsigned char* ptr;   // device address of g_noalloc_scratch on this device
};
constexpr int kNoAllocMaxDevices = 64;
static NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
static std::mutex g_noalloc_mu;

// Once per device, with that device current: the scratch's device address and the
// twiddle table of the fused kernel (no allocation).
static int noalloc_setup(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    cudaGetLastError();
    return fail(nullptr, DGDFT_CUDA_ERROR, "noalloc: no current CUDA device");
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocDevice& st = g_noalloc_dev[dev];
  if (!st.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return fail(nullptr, DGDFT_CUDA_ERROR, std::string("noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    }
    std::vector<float2> t32(kTwiddleCount);
    for (int n = 1; n <= kMaxLine; n++)
      for (int m = 0; m < n; m++) {
        const double a = -2.0 * M_PI * double(m) / double(n);
        t32[twiddle_offset(n) + m] = make_float2(float(std::cos(a)), float(std::sin(a)));
      }
    if (upload_fused_twiddles(t32.data())) {
      cudaGetLastError();
      return fail(nullptr, DGDFT_CUDA_ERROR, "noalloc: twiddle upload failed");
    }
    if (set_fused_smem_limits()) {
      cudaGetLastError();
      return fail(nullptr, DGDFT_CUDA_ERROR, "noalloc: shared-memory limit of the fused kernel not set");
    }
    st.ptr = static_cast<unsigned char*>(p);
    st.ready = true;
  }
  *out = st.ptr;
  return DGDFT_OK;
}

// bump placement inside the scratch (256-byte aligned pieces)
struct Bump {
  size_t used = 0;
  size_t take(size_t bytes) {
    const size_t off = (used + 255) & ~size_t(255);
    used = off + bytes;
    return off;
  }
};

}  // namespace dgdft

using namespace dgdft;

extern "C" int dgdft_apply_hamiltonian_noalloc(const dgdft_problem* prob, const dgdft_alb_params* prm, const float* X,
                                               float* Y, dgdft_stream stream) {
  if (!prob || !prm || !X || !Y) return fail(nullptr, DGDFT_INVALID_ARG, "noalloc: null argument");
  if (prm->precision != DGDFT_MIXED)
    return fail(nullptr, DGDFT_UNSUPPORTED, "noalloc: only the FP32 (DGDFT_MIXED) application is provided");
  Plan P;
  std::string msg;
  int r = build_plan(prob, prm, P, msg);
  if (r) return fail(nullptr, r, "noalloc: " + msg);
  for (const ShapeGroup& g : P.hx.groups)
    if (!g.fused_ok || !fused_shape_supported(g.qn))
      return fail(nullptr, DGDFT_UNSUPPORTED, "noalloc: a Q shape or its atom tables is outside the fused kernel");
  // scratch placement, checked against the fixed size before anything runs
  Bump b;
  const size_t o_desc = b.take(P.desc.size() * sizeof(ElemDesc));
  const size_t o_boxes = b.take(std::max<size_t>(1, P.boxes.size()) * sizeof(AtomBox));
  const size_t o_dtab = b.take(P.dtab.size() * sizeof(double));
  const size_t o_fat = b.take(std::max<size_t>(1, P.fatoms.size()) * sizeof(FusedAtomRec));
  const size_t nq = size_t(std::max(1, P.n_qboxes));
  const size_t o_plgw = b.take(nq * kProjCap * sizeof(uint2));
  const size_t o_pln = b.take(2 * nq * sizeof(int));
  const size_t o_xoff = b.take(P.off[OFF_X].size() * sizeof(long long));
  std::vector<size_t> o_grp(P.hx.groups.size());
  for (size_t i = 0; i < P.hx.groups.size(); i++) o_grp[i] = b.take(P.hx.groups[i].elems.size() * sizeof(int));
  const size_t o_flags = b.take(P.M * sizeof(int));
  const size_t o_v64 = b.take(P.tot[OFF_V] * sizeof(double));
  const size_t o_v32 = b.take(P.tot[OFF_V] * sizeof(float));
  if (b.used > kNoAllocScratchBytes)
    return fail(nullptr, DGDFT_UNSUPPORTED,
                "noalloc: the problem needs " + std::to_string(b.used) + " bytes of scratch, more than the fixed " +
                    std::to_string(kNoAllocScratchBytes) + " (24 MiB); use dgdft_apply_hamiltonian");
  unsigned char* base = nullptr;
  if ((r = noalloc_setup(&base))) return r;
  cudaStream_t st = (cudaStream_t)stream;
  auto up = [&](size_t off, const void* src, size_t bytes) {
    return bytes == 0 || cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  bool ok = up(o_desc, P.desc.data(), P.desc.size() * sizeof(ElemDesc)) &&
            up(o_boxes, P.boxes.data(), P.boxes.size() * sizeof(AtomBox)) &&
            up(o_dtab, P.dtab.data(), P.dtab.size() * sizeof(double)) &&
            up(o_fat, P.fatoms.data(), P.fatoms.size() * sizeof(FusedAtomRec)) &&
            up(o_xoff, P.off[OFF_X].data(), P.off[OFF_X].size() * sizeof(long long));
  for (size_t i = 0; ok && i < P.hx.groups.size(); i++) {
    ShapeGroup& g = P.hx.groups[i];
    ok = up(o_grp[i], g.elems.data(), g.elems.size() * sizeof(int));
    g.d_elems = reinterpret_cast<int*>(base + o_grp[i]);
    g.max_nvec = g.max_nblk;
  }
  ok = ok && cudaMemsetAsync(base + o_flags, 0, P.M * sizeof(int), st) == cudaSuccess;   // NaN flags start at 0
  if (!ok) {
    cudaGetLastError();
    return fail(nullptr, DGDFT_CUDA_ERROR, "noalloc: table upload failed");
  }
  const ElemDesc* d_desc = reinterpret_cast<const ElemDesc*>(base + o_desc);
  const AtomBox* d_boxes = reinterpret_cast<const AtomBox*>(base + o_boxes);
  double* V64 = reinterpret_cast<double*>(base + o_v64);
  float* V32 = reinterpret_cast<float*>(base + o_v32);
  g_max_points = P.max_points;
  g_max_nblk = P.max_nblk;
  g_max_nalb = P.max_nalb;
  BatchArgs ba{d_desc, nullptr, P.M};
  launch_setup_v(ba, d_boxes, reinterpret_cast<const double*>(base + o_dtab), prob->v_extra, P.r_cut, V64, V32,
                 reinterpret_cast<int*>(base + o_flags), st);
  HxArgs h{};
  h.desc = d_desc;
  h.flags = nullptr;
  h.boxes = d_boxes;
  h.dtab = reinterpret_cast<const double*>(base + o_dtab);
  h.xo = reinterpret_cast<const long long*>(base + o_xoff);
  h.so = nullptr;
  h.nvec_mode = NV_BLK;
  h.n_proj_per_atom = P.n_proj_per_atom;
  h.r_cut = P.r_cut;
  h.fatoms = reinterpret_cast<const FusedAtomRec*>(base + o_fat);
  h.plist = ProjList{reinterpret_cast<uint2*>(base + o_plgw), reinterpret_cast<int*>(base + o_pln)};
  if (P.n_qboxes > 0) launch_build_proj_lists(h.fatoms, h.dtab, P.n_qboxes, P.r_cut, h.plist, st);
  for (const ShapeGroup& g : P.hx.groups)
    if (!launch_fused_group(g, h, X, Y, nullptr, V32, nullptr, 0, OUT_APPLY, st))
      return fail(nullptr, DGDFT_UNSUPPORTED, "noalloc: fused kernel unavailable for a Q shape");
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(nullptr, DGDFT_CUDA_ERROR, std::string("noalloc: ") + cudaGetErrorString(e));
  // non-finite v_extra on some Q (flag set by the V_eff set-up): the output of that element is not valid
  std::vector<int> hf(P.M);
  e = cudaMemcpy(hf.data(), base + o_flags, P.M * sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(nullptr, DGDFT_CUDA_ERROR, std::string("noalloc: ") + cudaGetErrorString(e));
  for (int k = 0; k < P.M; k++)
    if (hf[k] & EF_BAD)
      return fail(nullptr, DGDFT_BAD_INPUT, "noalloc: element " + std::to_string(k) + ": v_extra is not finite on Q");
  return DGDFT_OK;
}
