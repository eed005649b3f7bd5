// Mixed-precision iHDG sweep loop: float64 defect correction around low-precision inner
// sweeps (see ihdg_mixed.h for the scheme).  The inner sweep is the same a1..a5 pass as the
// float64 one, on the correction equation, with low-precision storage of e and r and
// float32 arithmetic; its loop decision is a step-size test in the export space.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

#include "ihdg_kernels.h"
#include "ihdg_mixed.h"

namespace ihdg {

namespace {

cudaError_t mlaunch(MixedArgs& m, int which, int has_e, int count) {
  if (m.prec == IHDG_MIXED_BF16) return mixed_launch<__nv_bfloat16>(m, which, has_e, count);
  return mixed_launch<float>(m, which, has_e, count);
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

MixedLayout mixed_layout(const DevGeo& g, int prec) {
  MixedLayout L{};
  L.lp_bytes = prec == IHDG_MIXED_BF16 ? 2 : 4;
  // guard band of the correction arrays: the staged tensor-core kernel copies windows of 136
  // values starting up to one layer (the largest element-number step) plus 8 below an
  // element's number, and as far above it; the guards keep those windows inside the region
  // (what they read there lands only in masked rows)
  long long step = 1;
  for (int a = 0; a < g.dim; ++a) step = g.stride[a] > step ? g.stride[a] : step;
  L.pad = (step + 8 + 7) / 8 * 8 + 136;
  size_t one = a256((size_t)g.n_exp * g.ld * L.lp_bytes);
  size_t onep = a256(((size_t)g.n_exp * g.ld + 2 * (size_t)L.pad) * L.lp_bytes);
  L.rlp = 0;
  L.e0 = one;
  L.e1 = one + onep;
  L.lt = one + 2 * onep;
  L.total = one + 2 * onep + MIXED_LT_BYTES;   // + the register kernel's or the tensor-core kernel's operator
  return L;
}

void mixed_bind(MixedArgs& m, char* region, const MixedLayout& L, int prec) {
  m.prec = prec;
  m.E64 = m.base.ring + m.base.ring_stride;   // ring slots 1 and 2
  m.r64 = m.base.ring;                        // ring slot 0 (E^0 is dead once the outer loop runs)
  m.rlp = region + L.rlp;
  m.e[0] = region + L.e0 + (size_t)L.pad * L.lp_bytes;
  m.e[1] = region + L.e1 + (size_t)L.pad * L.lp_bytes;
  m.e_pad = L.pad;
  m.dLT = reinterpret_cast<float*>(region + L.lt);
}

ihdg_status run_mixed(Ctrl* hc, MixedArgs& m, const ihdg_options& o, const double** Eu, const double** Eu2,
                      const double** Et, const double** Et2, std::string& err, SweepTimer* tm) {
  const LaunchArgs& a = m.base;
  auto ck = [&](cudaError_t e, const char* where) {
    if (e != cudaSuccess) { err = std::string(where) + ": " + cudaGetErrorString(e); return false; }
    return true;
  };
  MixedArgs mm = m;
  int has_e = 0;
  // one launch, optionally timed with events; the timer gets the duration per sweep
  auto launch = [&](int which, int he, bool fp64) {
    if (tm->on && !ck(cudaEventRecord(tm->a, a.stream), "event")) return false;
    const int before = hc->iter;
    if (!ck(mlaunch(mm, which, he, 1), which == 0 ? "outer sweep kernel" : which == 1 ? "residual kernel" : "inner sweep kernel"))
      return false;
    m.ran = mm.ran;
    tm->launches += 1;
    if (!tm->on) return true;
    if (!ck(cudaEventRecord(tm->b, a.stream), "event") || !ck(cudaEventSynchronize(tm->b), "event") ||
        !ck(cudaMemcpy(hc, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost), "ctrl readback"))
      return false;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, tm->a, tm->b);
    const int n = which == 2 ? hc->iter - before : 1;
    if (fp64) { tm->fp64_ms += ms; tm->fp64_n += 1; }
    else if (n > 0) { tm->lowp_ms += ms; tm->lowp_n += n; }
    return true;
  };
  // Outer steps go out in batches (2, then 4) with one loop-state readback per batch: every
  // kernel returns at once when the loop has stopped (ctrl->done or ->timeout), so steps past
  // the last one cost only empty launches.  Profiling reads the state after every launch.
  int batch = tm->on ? 1 : 2;
  for (int outer = 0; outer < 1000000; outer += batch) {
    for (int b = 0; b < batch; ++b) {
      NvtxRange nv_outer("ihdg outer step");
      // the residual kernel (float64 norm of t(r), plus one low-precision sweep) is timed with
      // the float64 launches, so the low-precision figure is the persistent inner loop's alone
      if (!launch(0, has_e, true) || !launch(1, 0, true)) return IHDG_ERR_CUDA;
      has_e = 1;
      // the persistent inner kernel runs until the inner loop stops (it returns at once when
      // the residual check above already ended the solve)
      if (!launch(2, 0, false)) return IHDG_ERR_CUDA;
    }
    if (!ck(cudaMemcpyAsync(hc, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, a.stream), "ctrl readback") ||
        !ck(cudaStreamSynchronize(a.stream), "inner loop"))
      return IHDG_ERR_CUDA;
    if (hc->timeout) { err = "persistent inner sweep: a grid barrier wait ran out"; return IHDG_ERR_TIMEOUT; }
    if (hc->done) break;
    if (!tm->on && batch < 4) batch *= 2;
  }
  if (hc->outer == 0) {   // the first float64 sweep already met the tolerance (or failed)
    *Eu = a.ring;
    *Eu2 = nullptr;
    *Et = a.ring + a.ring_stride;
    *Et2 = nullptr;
    return IHDG_OK;
  }
  const double* Ecur = mm.E64 + (long long)(hc->outer & 1) * a.ring_stride;
  *Eu = Ecur;
  *Eu2 = nullptr;
  *Et = Ecur;
  *Et2 = mm.r64;
  return IHDG_OK;
}

}  // namespace ihdg
