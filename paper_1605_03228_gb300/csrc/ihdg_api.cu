// C-ABI of libihdg: argument checks, operator plans, workspace layout and the solve drivers.
// Every step of the iteration runs in the CUDA kernels of ihdg_kernels.cu / ihdg_mixed.cu;
// this file only validates, builds the float64 operators once per problem (host), moves
// data and decides when to launch.  There is no CPU fallback: without a device every
// entry point that computes fails with IHDG_ERR_CUDA.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <memory>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/ihdg.h"
#include "ihdg_dev.h"
#include "ihdg_kernels.h"
#include "ihdg_krylov.h"
#include "ihdg_mixed.h"
#include "ihdg_ops.h"
#include "ihdg_var.h"

using namespace ihdg;

namespace {

struct Plan {
  ihdg_mesh mesh{};
  ihdg_coeffs co{};
  Ops ops;
  std::vector<float> le32;   // host float32 copy of L_E (kernel parameter of the tile kernel)
  std::vector<double> img;   // packed float64 operator image
  std::vector<size_t> off;   // offsets of the operators in img
  DevGeo g{};
  OpsDev op{};
  void* dbuf = nullptr;
  size_t dbytes = 0;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool same_problem(const ihdg_mesh& a, const ihdg_mesh& b, const ihdg_coeffs& ca, const ihdg_coeffs& cb) {
  return std::memcmp(&a, &b, sizeof(ihdg_mesh)) == 0 && std::memcmp(&ca, &cb, sizeof(ihdg_coeffs)) == 0;
}

}  // namespace

namespace { struct Server; }

struct ihdg_ctx {
  int device = 0;
  std::string err;
  Server* server = nullptr;   // serving state (ihdg_server_start .. ihdg_server_stop)
  std::vector<std::unique_ptr<Plan>> plans;
  int plan_pin = 0;   // > 0: a call holds plan pointers, nothing is evicted
  // device scratch of the host-pointer calls (inputs, outputs, workspace)
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  Ctrl* h_ctrl = nullptr;   // pinned readback of the loop state
  // ihdg_autotune's choices: problem shape -> inner kernel, inner stopping ratio, sweeps per
  // grid barrier
  struct Tuned {
    int kernel;
    double rtol;
    int sps;
    int shape;   // tile shape of the temporally blocked kernel (1-based rank)
  };
  std::map<std::string, Tuned> tuned;
};

namespace {

ihdg_status fail(ihdg_ctx* c, ihdg_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}
ihdg_status cuda_fail(ihdg_ctx* c, cudaError_t e, const char* where) {
  std::ostringstream os;
  os << where << ": " << cudaGetErrorString(e);
  return fail(c, IHDG_ERR_CUDA, os.str());
}
#define CK(call, where)                                     \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

void fill_geo(const ihdg_mesh& m, const Ops& o, DevGeo& g) {
  std::memset(&g, 0, sizeof(g));
  g.dim = m.dim;
  g.nf = o.nf;
  g.nlf = o.nlf;
  g.n_in = o.n_in;
  g.n_exp = o.n_exp;
  g.nvol = o.nvol;
  g.nqv = o.nqv;
  g.nqf = o.nqf;
  g.nb = o.nb;
  g.n[0] = m.n[0];
  g.n[1] = m.n[1];
  g.n[2] = m.dim == 3 ? m.n[2] : 1;
  g.nel = (long long)g.n[0] * g.n[1] * g.n[2];
  g.ld = (g.nel + 31) / 32 * 32;
  g.stride[0] = 1;
  g.stride[1] = g.n[0];
  g.stride[2] = (long long)g.n[0] * g.n[1];
  g.nbf_off[0] = 0;
  g.nbf_off[1] = 2LL * g.n[1] * g.n[2];
  g.nbf_off[2] = g.nbf_off[1] + 2LL * g.n[0] * g.n[2];
  for (int f = 0; f < 6; ++f) {
    g.kind[f] = f < o.nlf ? o.face_kind[f] : 0;
    g.own_off[f] = o.own_off[f] < 0 ? 0 : o.own_off[f];
    g.nbr_off[f] = o.nbr_off[f] < 0 ? 0 : o.nbr_off[f];
  }
  g.bc_mirror = o.bc_mirror;
  g.steady = o.pde != IHDG_SWE;
  g.per_axis = o.layout_per_axis;
  g.live = 0ull;
  for (int f = 0; f < o.nlf; ++f)
    if (o.face_kind[f] == FK_OWN || o.face_kind[f] == FK_SUM)
      for (int j = 0; j < o.nf; ++j) g.live |= 1ull << (o.own_off[f] + j);
}

// Host part of a plan: float64 operators, device geometry, and the packed operator image
// (float64 block followed by the float32 copy of L_E) ready for one upload.
ihdg_status prepare_plan(ihdg_ctx* ctx, const ihdg_mesh& m, const ihdg_coeffs& co, Plan& pl) {
  pl.mesh = m;
  pl.co = co;
  std::string err;
  ihdg_status st = build_ops(m, co, pl.ops, err);
  if (st != IHDG_OK) return fail(ctx, st, err);
  const Ops& o = pl.ops;
  if (!shape_supported(m.dim, o.nf))
    return fail(ctx, IHDG_ERR_UNSUPPORTED, "this (dim, p) has no compiled sweep kernel (built: 2D p=1..4, 3D p=1..2)");
  fill_geo(m, o, pl.g);
  std::vector<double>& img = pl.img;
  std::vector<size_t>& off = pl.off;
  img.clear();
  off.clear();
  auto put = [&](const std::vector<double>& v) { off.push_back(img.size()); img.insert(img.end(), v.begin(), v.end()); size_t pad = (32 - img.size() % 32) % 32; img.insert(img.end(), pad, 0.0); };
  std::vector<double> Qp;
  for (int i = 0; i < o.n_in; ++i)
    for (int j = i; j < o.n_in; ++j) Qp.push_back(o.Q[i * o.n_in + j] * (i == j ? 1.0 : 2.0));
  std::vector<double> empty(1, 0.0);
  put(o.LE); put(Qp); put(o.Lvol); put(o.R); put(o.Mn);
  put(o.PF.empty() ? empty : o.PF); put(o.PV.empty() ? empty : o.PV);
  for (int f = 0; f < 6; ++f) put(o.PFb[f].empty() ? empty : o.PFb[f]);
  for (int f = 0; f < 6; ++f) put(o.PVb[f].empty() ? empty : o.PVb[f]);
  put(o.Pg.empty() ? empty : o.Pg);
  put(o.PqF.empty() ? empty : o.PqF); put(o.PqV.empty() ? empty : o.PqV);
  put(o.facevol);
  put(o.Mb);
  pl.le32.assign(o.LE.begin(), o.LE.end());
  pl.dbytes = align256(img.size() * sizeof(double)) + align256(pl.le32.size() * sizeof(float));
  return IHDG_OK;
}

// Copy the operator image to device memory at `base` (pl.dbytes bytes) on `stream` and point
// the plan's device operators into it.
ihdg_status upload_plan(ihdg_ctx* ctx, Plan& pl, void* base, cudaStream_t stream) {
  const size_t nd = pl.img.size();
  CK(cudaMemcpyAsync(base, pl.img.data(), nd * sizeof(double), cudaMemcpyHostToDevice, stream), "upload operators");
  float* d32 = reinterpret_cast<float*>(static_cast<char*>(base) + align256(nd * sizeof(double)));
  CK(cudaMemcpyAsync(d32, pl.le32.data(), pl.le32.size() * sizeof(float), cudaMemcpyHostToDevice, stream), "upload operators");
  CK(cudaStreamSynchronize(stream), "upload operators");
  const double* b = static_cast<const double*>(base);
  const std::vector<size_t>& off = pl.off;
  size_t k = 0;
  OpsDev& op = pl.op;
  op.LE = b + off[k++]; op.Qp = b + off[k++]; op.Lvol = b + off[k++]; op.R = b + off[k++]; op.Mn = b + off[k++];
  op.PF = b + off[k++]; op.PV = b + off[k++];
  for (int f = 0; f < 6; ++f) op.PFb[f] = b + off[k++];
  for (int f = 0; f < 6; ++f) op.PVb[f] = b + off[k++];
  op.Pg = b + off[k++]; op.PqF = b + off[k++]; op.PqV = b + off[k++]; op.facevol = b + off[k++];
  op.Mb = b + off[k++];
  for (int c = 0; c < 4; ++c) op.wcomp[c] = pl.ops.wcomp[c];
  op.LE32 = d32;
  return IHDG_OK;
}

// Build (or find) the plan of a problem: host float64 operators and their device copies
// (cudaMalloc'd, cached in the context).
ihdg_status get_plan(ihdg_ctx* ctx, const ihdg_mesh& m, const ihdg_coeffs& co, Plan*& out, double* setup_ms) {
  for (auto& p : ctx->plans)
    if (same_problem(p->mesh, m, p->co, co)) { out = p.get(); if (setup_ms) *setup_ms = 0.0; return IHDG_OK; }
  auto t0 = std::chrono::steady_clock::now();
  auto pl = std::make_unique<Plan>();
  ihdg_status st = prepare_plan(ctx, m, co, *pl);
  if (st != IHDG_OK) return st;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(cudaMalloc(&pl->dbuf, pl->dbytes), "cudaMalloc(operators)");
  st = upload_plan(ctx, *pl, pl->dbuf, nullptr);
  if (st != IHDG_OK) {
    cudaFree(pl->dbuf);
    return st;
  }
  while (ctx->plans.size() >= 16 && ctx->plan_pin == 0) {
    cudaFree(ctx->plans.front()->dbuf);
    ctx->plans.erase(ctx->plans.begin());
  }
  out = pl.get();
  ctx->plans.push_back(std::move(pl));
  if (setup_ms) *setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return IHDG_OK;
}

// Workspace layout of one solve (offsets in bytes from the workspace base).
struct Layout {
  size_t ctrl, partials, res_hist, F, V, ring, qnext, mixed, kry, total;
  MixedLayout mx;
};

Layout layout_for(const DevGeo& g, const ihdg_options& o, bool swe) {
  Layout L{};
  size_t at = 0;
  auto take = [&](size_t bytes) { size_t r = at; at += align256(bytes); return r; };
  int maxit = o.max_iters > 0 ? o.max_iters : 2000;
  L.ctrl = take(sizeof(Ctrl));
  L.partials = take(sizeof(double) * (size_t)partials_needed(g.nel));
  L.res_hist = take(sizeof(double) * (size_t)(maxit + 2));
  L.F = take(sizeof(double) * (size_t)g.n_exp * g.ld);
  L.V = take(sizeof(double) * (size_t)g.nvol * g.ld);
  L.ring = take(3 * sizeof(double) * (size_t)g.n_exp * g.ld);
  L.qnext = swe ? take(sizeof(double) * (size_t)g.nvol * g.nel) : 0;
  if (o.prec != IHDG_FP64) {
    L.mx = mixed_layout(g, o.prec);
    L.mixed = take(L.mx.total);
  }
  if (o.krylov_restart > 0) L.kry = take(krylov_bytes((long long)g.n_exp * g.ld, o.krylov_restart));
  L.total = at;
  return L;
}

ihdg_options defaults(const ihdg_options* o) {
  ihdg_options r{};
  if (o) r = *o;
  if (r.max_iters <= 0) r.max_iters = 2000;
  if (r.diverge_factor == 0.0) r.diverge_factor = 1e6;
  if (r.inner_max <= 0) r.inner_max = 400;
  // Inner stop well above the low-precision rounding floor: an inner loop pushed towards its
  // floor spends sweeps without progress, while the float64 outer step that follows restores
  // full accuracy.  Measured on the conv.-diff., 3D transport and shallow-water workloads
  // (total sweeps to tol fell by 20-75% against 1e-4 / 1e-2).
  if (r.inner_rtol < 0.0) r.inner_rtol = 0.0;   // 0: automatic, resolved with the inner kernel
  return r;
}

ihdg_status check_opts(ihdg_ctx* ctx, const ihdg_options& o) {
  if (!(o.tol >= 0.0) || !std::isfinite(o.tol)) return fail(ctx, IHDG_ERR_INVALID, "opts.tol must be finite and >= 0");
  if (o.prec < IHDG_FP64 || o.prec > IHDG_MIXED_BF16) return fail(ctx, IHDG_ERR_INVALID, "opts.prec is not a known precision");
  if (o.max_iters > 100000000) return fail(ctx, IHDG_ERR_INVALID, "opts.max_iters too large");
  if (o.sweeps_per_sync < 0 || o.sweeps_per_sync > 8)
    return fail(ctx, IHDG_ERR_INVALID, "opts.sweeps_per_sync must be in 0..8");
  if (o.tile_shape < 0 || o.tile_shape > 64) return fail(ctx, IHDG_ERR_INVALID, "opts.tile_shape must be in 0..64");
  if (o.krylov_restart < 0 || o.krylov_restart > 4096)
    return fail(ctx, IHDG_ERR_INVALID, "opts.krylov_restart must be in 0..4096");
  if (o.krylov_restart > 0 && o.prec != IHDG_FP64)
    return fail(ctx, IHDG_ERR_INVALID, "opts.krylov_restart needs opts.prec = IHDG_FP64");
  if (o.inner_kernel < IHDG_KERNEL_AUTO || o.inner_kernel > IHDG_KERNEL_GLOBAL)
    return fail(ctx, IHDG_ERR_INVALID, "opts.inner_kernel is not a known kernel");
  return IHDG_OK;
}

// Key of ihdg_autotune's cache: the problem shape and precision.
std::string tune_key(const ihdg_mesh& m, const ihdg_coeffs& c, int prec) {
  std::ostringstream os;
  os << c.pde << '/' << c.flux << '/' << m.dim << '/' << m.n[0] << 'x' << m.n[1] << 'x' << (m.dim == 3 ? m.n[2] : 1)
     << "/p" << m.p << "/prec" << prec;
  return os.str();
}

// One solve of the iteration on the device: forcing, first sweep, sweep loop (float64 or
// mixed), reconstruction of u^K and the trace.  `u0` (device, may be null) is the initial
// guess; for shallow water src.q holds q^m and u0 == src.q (warm start).
ihdg_status device_iterate(ihdg_ctx* ctx, Plan* pl, const ihdg_options& o, const SrcDev& src, const double* u0,
                           double* d_u, double* d_tr, char* ws, const Layout& L, cudaStream_t stream,
                           ihdg_result* res) {
  NvtxRange nv_solve(o.prec == IHDG_FP64 ? "ihdg solve (float64)" : "ihdg solve (mixed)");
  LaunchArgs a{};
  a.g = pl->g;
  a.op = pl->op;
  a.src = src;
  a.u0 = u0;
  a.F = reinterpret_cast<double*>(ws + L.F);
  a.V = reinterpret_cast<double*>(ws + L.V);
  a.ring = reinterpret_cast<double*>(ws + L.ring);
  a.ring_stride = (long long)pl->g.n_exp * pl->g.ld;
  a.ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
  a.partials = reinterpret_cast<double*>(ws + L.partials);
  a.res_hist = reinterpret_cast<double*>(ws + L.res_hist);
  a.stream = stream;
  int inner_used = 0;
  // every event this call creates is destroyed on every return path (errors included)
  struct Events {
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    ~Events() {
      for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    }
  } evs;
  CK(cudaEventCreate(&evs.ev[0]), "cudaEventCreate");
  CK(cudaEventCreate(&evs.ev[1]), "cudaEventCreate");
  cudaEvent_t e0 = evs.ev[0], e1 = evs.ev[1];
  CK(cudaEventRecord(e0, stream), "cudaEventRecord");
  SweepTimer tm;
  tm.on = o.profile != 0;
  if (tm.on) {
    CK(cudaEventCreate(&evs.ev[2]), "cudaEventCreate");
    CK(cudaEventCreate(&evs.ev[3]), "cudaEventCreate");
    tm.a = evs.ev[2];
    tm.b = evs.ev[3];
  }
  // inner kernel and stopping ratio of the mixed path: the caller's, else the autotuned ones
  // for this problem shape, else the automatic rules
  int inner_kernel = o.inner_kernel;
  double inner_rtol = o.inner_rtol;
  int sps = o.sweeps_per_sync;
  int shape = o.tile_shape;
  if (o.prec != IHDG_FP64 && inner_kernel == IHDG_KERNEL_AUTO && inner_rtol <= 0.0 && sps <= 0 && shape <= 0) {
    auto it = ctx->tuned.find(tune_key(pl->mesh, pl->co, o.prec));
    if (it != ctx->tuned.end()) {
      inner_kernel = it->second.kernel;
      inner_rtol = it->second.rtol;
      sps = it->second.sps;
      shape = it->second.shape;
    }
  }
  // Inner stop well above the low-precision rounding floor: an inner loop pushed towards its
  // floor spends sweeps without progress, while the float64 outer step that follows restores
  // full accuracy (measured on the conv.-diff., 3D transport and shallow-water workloads).
  if (inner_rtol <= 0.0) inner_rtol = o.prec == IHDG_MIXED_BF16 ? 0.2 : (o.prec == IHDG_MIXED_TF32 ? 1e-2 : 2e-3);
  // Bound of every grid-barrier wait (~1 s of SM clock) and, for the failure-detection tests
  // only, a block that never arrives (IHDG_TEST_STALL_BLOCK) with a shorter bound
  // (IHDG_TEST_WAIT_CYCLES): the waits then run out and the call returns IHDG_ERR_TIMEOUT.
  long long wait_cycles = 2000000000LL;
  int stall_block = -1;
  if (const char* w = std::getenv("IHDG_TEST_WAIT_CYCLES")) {
    const long long v = std::atoll(w);
    if (v > 0) wait_cycles = v;
  }
  if (const char* b = std::getenv("IHDG_TEST_STALL_BLOCK")) stall_block = std::atoi(b);
  CK(launch_ctrl_init(a, o.tol, o.diverge_factor, o.max_iters, o.inner_max, inner_rtol, wait_cycles, stall_block),
     "ctrl init");
  CK(launch_forcing(a), "forcing kernel");
  tm.launches += 2;
  Ctrl* hc = ctx->h_ctrl;
  bool mixed = o.prec != IHDG_FP64;
  const bool kry = o.krylov_restart > 0;
  KryOut ko;
  const double* Eu = nullptr;     // exports whose traces fed the final local solve
  const double* Eu2 = nullptr;    //   (+ a second array, added; mixed path)
  const double* Et = nullptr;     // exports of u^K
  const double* Et2 = nullptr;
  if (kry) {
    // GMRES around the sweep on (I - T) E = F from E^0 = the exports of u0 (or zero); the
    // solution is a fixed point of the sweep, so its exports feed both the final local solve
    // and the trace
    NvtxRange nv_kry("ihdg GMRES");
    double* Ex = a.ring;
    CK(cudaMemsetAsync(Ex, 0, sizeof(double) * (size_t)a.ring_stride, stream), "memset");
    if (u0) { CK(launch_export0(a, u0, Ex), "initial export kernel"); tm.launches += 1; }
    if (run_krylov(a, o.krylov_restart, o.tol, o.max_iters, Ex, a.ring + a.ring_stride, ws + L.kry, &ko, ctx->err) !=
        cudaSuccess)
      return fail(ctx, IHDG_ERR_CUDA, ctx->err);
    tm.launches += ko.launches;
    Eu = Ex;
    Et = Ex;
  } else {
    CK(launch_export0(a, u0, a.ring), "initial export kernel");
    CK(launch_first(a), "first sweep kernel");
    tm.launches += 2;
  }
  if (!kry && !mixed) {
    // the whole loop in one cooperative launch when its grid is co-resident (not in profile
    // mode, which times every sweep launch); otherwise, or after it, batches of launches
    if (!tm.on) {
      cudaError_t pe = launch_sweep64_persist(a);
      if (pe == cudaSuccess) {
        tm.launches += 1;
        CK(cudaMemcpyAsync(hc, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream), "ctrl readback");
        CK(cudaStreamSynchronize(stream), "persistent sweep loop");
        if (hc->timeout) return fail(ctx, IHDG_ERR_TIMEOUT, "persistent float64 sweep: a grid barrier wait ran out");
      } else if (pe != cudaErrorNotSupported) {
        return cuda_fail(ctx, pe, "persistent sweep kernel");
      } else {
        cudaGetLastError();
      }
    }
    int batch = 2;
    for (;;) {
      CK(cudaMemcpyAsync(hc, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream), "ctrl readback");
      CK(cudaStreamSynchronize(stream), "sweep loop");
      if (hc->done) break;
      int left = hc->max_iters - hc->iter;
      int n = batch < left ? batch : left;
      if (n <= 0) break;
      if (tm.on) {
        CK(cudaEventRecord(tm.a, stream), "cudaEventRecord");
        CK(launch_sweep64(a, 1), "sweep kernel");
        CK(cudaEventRecord(tm.b, stream), "cudaEventRecord");
        CK(cudaEventSynchronize(tm.b), "sweep kernel");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, tm.a, tm.b);
        tm.fp64_ms += ms;
        tm.fp64_n += 1;
        tm.launches += 1;
        continue;
      }
      CK(launch_sweep64(a, n), "sweep kernel");
      tm.launches += n;
      if (batch < 32) batch *= 2;
    }
    int K = hc->iter;
    Et = a.ring + (long long)(K % 3) * a.ring_stride;
    Eu = a.ring + (long long)((K + 2) % 3) * a.ring_stride;
  } else if (!kry) {
    MixedArgs m{};
    m.base = a;
    mixed_bind(m, ws + L.mixed, L.mx, o.prec);
    // IHDG_PERSISTENT_GRID caps the persistent kernel's grid (tuning and grid-stride tests)
    if (const char* cap = std::getenv("IHDG_PERSISTENT_GRID")) {
      int v = std::atoi(cap);
      if (v > 0) m.max_grid = v;
    }
    // Inner sweeps run their local apply on the tensor cores (tcgen05) by default for bf16,
    // tf32, and float32 on 3D meshes (split tf32, three passes); float32 on 2D meshes uses the
    // register kernel.  IHDG_INNER_KERNEL overrides: "tc" (tensor cores wherever the shape
    // fits), "tile" (register- or shared-memory-resident CUDA-core kernels) or "global".
    m.use_tc = (o.prec == IHDG_MIXED_BF16 || o.prec == IHDG_MIXED_TF32 || (o.prec == IHDG_MIXED_FP32 && pl->g.dim == 3)) ? 1 : 0;
    if (inner_kernel != IHDG_KERNEL_AUTO) {
      m.use_tc = inner_kernel == IHDG_KERNEL_TENSOR_CORES ? 1 : 0;
      m.no_tile = inner_kernel == IHDG_KERNEL_GLOBAL ? 1 : 0;
    } else if (const char* ker = std::getenv("IHDG_INNER_KERNEL")) {
      m.no_tile = std::strcmp(ker, "global") == 0;
      m.use_tc = std::strcmp(ker, "tc") == 0 ? 1 : 0;
    }
    // IHDG_REG_NT=512: register kernel with two 512-thread blocks per SM instead of one
    // 1024-thread block (twice the grid-barrier arrivals; 1.4% slower on the headline mesh)
    if (const char* nt = std::getenv("IHDG_REG_NT")) m.reg_nt = std::atoi(nt) == 512 ? 512 : 1024;
    // IHDG_TILE_LPE=1 skips the register-resident 2D kernel (one element per thread instead)
    if (const char* lpe = std::getenv("IHDG_TILE_LPE")) m.tile_lpe = std::atoi(lpe) == 1 ? 1 : 4;
    // sweeps per grid barrier of the 2D CUDA-core inner kernel (temporal blocking when >= 2);
    // IHDG_SWEEPS_PER_SYNC overrides the automatic choice, 4 (measured on the 256^2 p=3
    // conv.-diff. solve: 3.2 us per sweep against 4.8 with one barrier per sweep)
    if (sps <= 0)
      if (const char* h = std::getenv("IHDG_SWEEPS_PER_SYNC")) sps = std::atoi(h);
    if (sps <= 0) sps = 4;
    m.blk_h = sps >= 2 ? (sps > 8 ? 8 : sps) : 0;
    m.blk_rank = shape >= 1 ? shape - 1 : 0;
    m.LE32h = pl->le32.data();
    m.slots = partials_needed(pl->g.nel);
    ihdg_status st = run_mixed(ctx->h_ctrl, m, o, &Eu, &Eu2, &Et, &Et2, ctx->err, &tm);
    if (st != IHDG_OK) return fail(ctx, st, ctx->err);
    inner_used = m.ran;
  }
  if (d_u) { CK(launch_reconstruct(a, Eu, Eu2, d_u), "reconstruct kernel"); tm.launches += 1; }
  if (d_tr) {
    double beta[3] = {pl->co.beta[0], pl->co.beta[1], pl->co.beta[2]};
    long long nface = count_faces(pl->mesh, nullptr);
    CK(launch_trace_out(a, Et, Et2, d_u, (int)pl->co.pde, beta, pl->ops.alpha_axis, nface, d_tr), "trace kernel");
    tm.launches += 1;
  }
  CK(cudaEventRecord(e1, stream), "cudaEventRecord");
  CK(cudaMemcpyAsync(hc, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream), "ctrl readback");
  CK(cudaStreamSynchronize(stream), "solve");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  if (res) {
    res->fp64_sweep_ms = tm.fp64_n ? tm.fp64_ms / tm.fp64_n : 0.0;
    res->lowp_sweep_ms = tm.lowp_n ? tm.lowp_ms / tm.lowp_n : 0.0;
    res->fp64_launches = tm.fp64_n;
    res->lowp_launches = tm.lowp_n;
    res->kernel_launches = tm.launches;
    res->iterations = hc->iter;
    res->fp64_sweeps = hc->fp64_sweeps;
    res->lowp_sweeps = hc->lowp_sweeps;
    res->residual = hc->res;
    res->status = (ihdg_status)hc->status;
    res->solve_ms = ms;
    res->inner_kernel_used = inner_used;
    if (kry) {
      res->iterations = ko.iters;
      res->fp64_sweeps = ko.iters;
      res->lowp_sweeps = 0;
      res->residual = ko.res_true;
      res->status = (ihdg_status)ko.status;
    }
  }
  return IHDG_OK;
}

ihdg_status ensure_scratch(ihdg_ctx* ctx, size_t bytes) {
  if (ctx->scratch_bytes >= bytes) return IHDG_OK;
  if (ctx->scratch) cudaFree(ctx->scratch);
  ctx->scratch = nullptr;
  ctx->scratch_bytes = 0;
  cudaError_t e = cudaMalloc(&ctx->scratch, bytes);
  if (e != cudaSuccess) return fail(ctx, IHDG_ERR_NOMEM, std::string("device scratch allocation failed: ") + cudaGetErrorString(e));
  ctx->scratch_bytes = bytes;
  return IHDG_OK;
}

}  // namespace

extern "C" {

ihdg_status ihdg_create(ihdg_ctx** out, int device) {
  if (!out) return IHDG_ERR_INVALID;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return IHDG_ERR_CUDA;
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, device) != cudaSuccess) return IHDG_ERR_CUDA;
  if (pr.major != 10 || pr.minor != 3) return IHDG_ERR_CUDA;   // built for sm_103a only
  auto* c = new ihdg_ctx();
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess || cudaMallocHost(&c->h_ctrl, sizeof(Ctrl)) != cudaSuccess) {
    delete c;
    return IHDG_ERR_CUDA;
  }
  *out = c;
  return IHDG_OK;
}

void ihdg_destroy(ihdg_ctx* ctx) {
  if (!ctx) return;
  if (ctx->server) ihdg_server_stop(ctx);
  cudaSetDevice(ctx->device);
  for (auto& p : ctx->plans) cudaFree(p->dbuf);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->h_ctrl) cudaFreeHost(ctx->h_ctrl);
  delete ctx;
}

const char* ihdg_last_error(const ihdg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

ihdg_status ihdg_abi_sizes(size_t* out, int n) {
  if (!out || n < 0) return IHDG_ERR_INVALID;
  const size_t sz[6] = {sizeof(ihdg_mesh), sizeof(ihdg_coeffs), sizeof(ihdg_options),
                        sizeof(ihdg_result), sizeof(ihdg_sizes), sizeof(ihdg_peaks)};
  for (int i = 0; i < n && i < 6; ++i) out[i] = sz[i];
  return IHDG_OK;
}

ihdg_status ihdg_problem_sizes(const ihdg_mesh* mesh, const ihdg_coeffs* co, ihdg_sizes* out) {
  if (!mesh || !co || !out) return IHDG_ERR_INVALID;
  std::string err;
  Ops o;
  ihdg_status st = build_ops(*mesh, *co, o, err);
  if (st != IHDG_OK) return st;
  std::memset(out, 0, sizeof(*out));
  out->n_el = 1;
  for (int a = 0; a < mesh->dim; ++a) out->n_el *= mesh->n[a];
  out->nvol = o.nvol;
  out->ncomp = o.ncomp;
  out->nqv = co->pde == IHDG_SWE ? 0 : o.nqv;
  out->nqf = co->pde == IHDG_SWE ? 0 : o.nqf;
  out->n_face = count_faces(*mesh, &out->n_bface);
  out->nface_nodes = o.nf;
  out->n_exp = o.n_exp;
  out->n_in = o.n_in;
  return IHDG_OK;
}

ihdg_status ihdg_quadrature_points(const ihdg_mesh* mesh, double* vol_xyz, double* bnd_xyz) {
  if (!mesh) return IHDG_ERR_INVALID;
  std::string err;
  ihdg_status st = validate(*mesh, nullptr, err);
  if (st != IHDG_OK) return st;
  quadrature_points(*mesh, vol_xyz, bnd_xyz);
  return IHDG_OK;
}

ihdg_status ihdg_node_points(const ihdg_mesh* mesh, double* xyz) {
  if (!mesh || !xyz) return IHDG_ERR_INVALID;
  std::string err;
  ihdg_status st = validate(*mesh, nullptr, err);
  if (st != IHDG_OK) return st;
  node_points(*mesh, xyz);
  return IHDG_OK;
}

ihdg_status ihdg_workspace_bytes(const ihdg_mesh* mesh, const ihdg_coeffs* co, const ihdg_options* opts, size_t* bytes) {
  if (!mesh || !co || !bytes) return IHDG_ERR_INVALID;
  if (opts && (opts->krylov_restart < 0 || opts->krylov_restart > 4096)) return IHDG_ERR_INVALID;
  std::string err;
  Ops o;
  ihdg_status st = build_ops(*mesh, *co, o, err);
  if (st != IHDG_OK) return st;
  DevGeo g;
  fill_geo(*mesh, o, g);
  *bytes = layout_for(g, defaults(opts), co->pde == IHDG_SWE).total;
  return IHDG_OK;
}

ihdg_status ihdg_solve_device(ihdg_ctx* ctx, const ihdg_mesh* mesh, const ihdg_coeffs* co, const double* d_f,
                              const double* d_g, const ihdg_options* opts, double* d_u, double* d_tr,
                              void* d_ws, size_t ws_bytes, void* stream, ihdg_result* res) {
  if (!ctx) return IHDG_ERR_INVALID;
  if (!mesh || !co || !d_f || !d_g || !d_ws || !d_u) return fail(ctx, IHDG_ERR_INVALID, "null argument");
  if (co->pde == IHDG_SWE) return fail(ctx, IHDG_ERR_INVALID, "shallow water is solved by ihdg_swe_steps*");
  if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0) return fail(ctx, IHDG_ERR_INVALID, "workspace must be 256-byte aligned");
  ihdg_options o = defaults(opts);
  ihdg_status st = check_opts(ctx, o);
  if (st != IHDG_OK) return st;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  Plan* pl = nullptr;
  double setup_ms = 0.0;
  st = get_plan(ctx, *mesh, *co, pl, &setup_ms);
  if (st != IHDG_OK) return st;
  Layout L = layout_for(pl->g, o, false);
  if (ws_bytes < L.total) return fail(ctx, IHDG_ERR_NOMEM, "workspace smaller than ihdg_workspace_bytes()");
  SrcDev src{d_f, d_g, nullptr};
  st = device_iterate(ctx, pl, o, src, o.u0, d_u, d_tr, static_cast<char*>(d_ws), L, static_cast<cudaStream_t>(stream), res);
  if (st != IHDG_OK) return st;
  if (res) res->setup_ms = setup_ms;
  ctx->err.clear();
  return IHDG_OK;
}

ihdg_status ihdg_solve(ihdg_ctx* ctx, const ihdg_mesh* mesh, const ihdg_coeffs* co, const double* f_qp,
                       const double* g_qp, const ihdg_options* opts, double* u_out, double* trace_out,
                       ihdg_result* res) {
  if (!ctx) return IHDG_ERR_INVALID;
  if (!mesh || !co || !f_qp || !g_qp || !u_out) return fail(ctx, IHDG_ERR_INVALID, "null argument");
  if (co->pde == IHDG_SWE) return fail(ctx, IHDG_ERR_INVALID, "shallow water is solved by ihdg_swe_steps*");
  ihdg_sizes sz;
  ihdg_status st = ihdg_problem_sizes(mesh, co, &sz);
  if (st != IHDG_OK) {
    std::string err;
    validate(*mesh, co, err);
    return fail(ctx, st, err.empty() ? "invalid problem" : err);
  }
  ihdg_options o = defaults(opts);
  st = check_opts(ctx, o);
  if (st != IHDG_OK) return st;
  size_t ws = 0;
  ihdg_workspace_bytes(mesh, co, &o, &ws);
  size_t bf = align256(sizeof(double) * sz.n_el * sz.nqv), bg = align256(sizeof(double) * sz.n_bface * sz.nqf);
  size_t bu = align256(sizeof(double) * sz.n_el * sz.nvol), bt = align256(sizeof(double) * sz.n_face * sz.nface_nodes);
  size_t bu0 = o.u0 ? bu : 0;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  st = ensure_scratch(ctx, bf + bg + bu + bt + bu0 + ws);
  if (st != IHDG_OK) return st;
  char* s = static_cast<char*>(ctx->scratch);
  double* d_f = reinterpret_cast<double*>(s);
  double* d_g = reinterpret_cast<double*>(s + bf);
  double* d_u = reinterpret_cast<double*>(s + bf + bg);
  double* d_t = reinterpret_cast<double*>(s + bf + bg + bu);
  double* d_u0 = o.u0 ? reinterpret_cast<double*>(s + bf + bg + bu + bt) : nullptr;
  char* d_ws = s + bf + bg + bu + bt + bu0;
  cudaStream_t stream = nullptr;
  CK(cudaMemcpyAsync(d_f, f_qp, sizeof(double) * sz.n_el * sz.nqv, cudaMemcpyHostToDevice, stream), "copy f");
  CK(cudaMemcpyAsync(d_g, g_qp, sizeof(double) * sz.n_bface * sz.nqf, cudaMemcpyHostToDevice, stream), "copy g");
  if (o.u0) CK(cudaMemcpyAsync(d_u0, o.u0, sizeof(double) * sz.n_el * sz.nvol, cudaMemcpyHostToDevice, stream), "copy u0");
  ihdg_options od = o;
  od.u0 = d_u0;
  st = ihdg_solve_device(ctx, mesh, co, d_f, d_g, &od, d_u, trace_out ? d_t : nullptr, d_ws, ws, stream, res);
  if (st != IHDG_OK) return st;
  CK(cudaMemcpy(u_out, d_u, sizeof(double) * sz.n_el * sz.nvol, cudaMemcpyDeviceToHost), "copy u");
  if (trace_out) CK(cudaMemcpy(trace_out, d_t, sizeof(double) * sz.n_face * sz.nface_nodes, cudaMemcpyDeviceToHost), "copy trace");
  return IHDG_OK;
}

ihdg_status ihdg_autotune(ihdg_ctx* ctx, const ihdg_mesh* mesh, const ihdg_coeffs* co, const double* f_qp,
                          const double* g_qp, const ihdg_options* opts, ihdg_options* tuned, double* best_ms) {
  NvtxRange nv_tune("ihdg autotune");
  if (!ctx) return IHDG_ERR_INVALID;
  if (!mesh || !co || !f_qp || !g_qp || !tuned) return fail(ctx, IHDG_ERR_INVALID, "null argument");
  if (co->pde == IHDG_SWE) return fail(ctx, IHDG_ERR_INVALID, "shallow water is solved by ihdg_swe_steps*");
  ihdg_sizes sz;
  ihdg_status st = ihdg_problem_sizes(mesh, co, &sz);
  if (st != IHDG_OK) {
    std::string err;
    validate(*mesh, co, err);
    return fail(ctx, st, err.empty() ? "invalid problem" : err);
  }
  ihdg_options o = defaults(opts);
  st = check_opts(ctx, o);
  if (st != IHDG_OK) return st;
  *tuned = opts ? *opts : o;
  if (best_ms) *best_ms = 0.0;
  if (o.prec == IHDG_FP64) return IHDG_OK;
  size_t ws = 0;
  ihdg_workspace_bytes(mesh, co, &o, &ws);
  size_t bf = align256(sizeof(double) * sz.n_el * sz.nqv), bg = align256(sizeof(double) * sz.n_bface * sz.nqf);
  size_t bu = align256(sizeof(double) * sz.n_el * sz.nvol);
  size_t bu0 = o.u0 ? bu : 0;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  st = ensure_scratch(ctx, bf + bg + bu + bu0 + ws);
  if (st != IHDG_OK) return st;
  char* s = static_cast<char*>(ctx->scratch);
  double* d_f = reinterpret_cast<double*>(s);
  double* d_g = reinterpret_cast<double*>(s + bf);
  double* d_u = reinterpret_cast<double*>(s + bf + bg);
  double* d_u0 = o.u0 ? reinterpret_cast<double*>(s + bf + bg + bu) : nullptr;
  char* d_ws = s + bf + bg + bu + bu0;
  CK(cudaMemcpy(d_f, f_qp, sizeof(double) * sz.n_el * sz.nqv, cudaMemcpyHostToDevice), "copy f");
  CK(cudaMemcpy(d_g, g_qp, sizeof(double) * sz.n_bface * sz.nqf, cudaMemcpyHostToDevice), "copy g");
  if (o.u0) CK(cudaMemcpy(d_u0, o.u0, sizeof(double) * sz.n_el * sz.nvol, cudaMemcpyHostToDevice), "copy u0");
  static const double ladder32[] = {5e-4, 1e-3, 2e-3, 5e-3, 1e-2};
  static const double ladder16[] = {2e-2, 5e-2, 0.1, 0.2, 0.3};
  const double* ladder = o.prec == IHDG_MIXED_BF16 ? ladder16 : ladder32;
  const int kernels[] = {IHDG_KERNEL_TENSOR_CORES, IHDG_KERNEL_CUDA_CORES};
  // sweeps per grid barrier: the temporally blocked CUDA-core kernel exists for 2D meshes
  const int sps_2d[] = {1, 2, 3, 4};
  const int sps_1[] = {1};
  // tile shapes of the temporally blocked kernel: the three of smallest tile + halo area
  constexpr int NSHAPE = 3;
  double best = 1e300;
  int best_k = IHDG_KERNEL_AUTO, best_s = 1, best_shape = 1;
  double best_r = 0.0;
  for (int pass = 0; pass < 2; ++pass)          // pass 0 warms every kernel up (module loads)
    for (int k : kernels) {
      const bool blk = k == IHDG_KERNEL_CUDA_CORES && mesh->dim == 2;
      const int* sl = blk ? sps_2d : sps_1;
      const int ns = blk ? 4 : 1;
      for (int si = 0; si < ns; ++si)
        for (int shape = 1; shape <= (sl[si] >= 2 ? NSHAPE : 1); ++shape)
          for (int i = 0; i < (pass == 0 ? 1 : 5); ++i) {
            ihdg_options oc = o;
            oc.u0 = d_u0;
            oc.inner_kernel = static_cast<ihdg_inner_kernel>(k);
            oc.inner_rtol = ladder[pass == 0 ? 2 : i];
            oc.sweeps_per_sync = sl[si];
            oc.tile_shape = shape;
            oc.profile = 0;
            ihdg_result r{};
            st = ihdg_solve_device(ctx, mesh, co, d_f, d_g, &oc, d_u, nullptr, d_ws, ws, nullptr, &r);
            if (st == IHDG_ERR_CUDA || st == IHDG_ERR_TIMEOUT || st == IHDG_ERR_NOMEM) return st;
            if (pass == 0 || st != IHDG_OK || r.status != IHDG_OK) continue;
            if (r.solve_ms < best) {
              best = r.solve_ms;
              best_k = k;
              best_r = oc.inner_rtol;
              best_s = sl[si];
              best_shape = shape;
            }
          }
    }
  if (best_k == IHDG_KERNEL_AUTO) return fail(ctx, IHDG_NOT_CONVERGED, "no candidate converged");
  ctx->tuned[tune_key(*mesh, *co, o.prec)] = {best_k, best_r, best_s, best_shape};
  tuned->inner_kernel = static_cast<ihdg_inner_kernel>(best_k);
  tuned->inner_rtol = best_r;
  tuned->sweeps_per_sync = best_s;
  tuned->tile_shape = best_shape;
  if (best_ms) *best_ms = best;
  ctx->err.clear();
  return IHDG_OK;
}

// ---------------------------------------------------------------------------------------
// Solve that allocates no device memory.  Its scratch (operator image and the whole solve
// workspace) is this file-scope array, which every GPU that loads the library holds until
// the process exits.  Host code cannot use the array's name as a device address: the first
// call on each device resolves the address with cudaGetSymbolAddress (with that device
// current) and every call passes that pointer on.  All calls share the array, so calls whose
// work overlaps on the GPU (other streams, other host threads) race; each call writes every
// scratch value before reading it (the loop state is initialised by its first kernel).
static __device__ __align__(256) unsigned char g_ihdg_static_scratch[IHDG_STATIC_SCRATCH_BYTES];

namespace {
std::mutex g_static_mu;
void* g_static_addr[256] = {nullptr};   // device address of g_ihdg_static_scratch, per device

ihdg_status static_scratch(ihdg_ctx* ctx, void** out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (ctx->device < 0 || ctx->device >= 256) return fail(ctx, IHDG_ERR_INVALID, "device index out of range");
  if (!g_static_addr[ctx->device]) {
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_ihdg_static_scratch), "cudaGetSymbolAddress(static scratch)");
    g_static_addr[ctx->device] = p;
  }
  *out = g_static_addr[ctx->device];
  return IHDG_OK;
}
}  // namespace

extern "C" ihdg_status ihdg_solve_device_static(ihdg_ctx* ctx, const ihdg_mesh* mesh, const ihdg_coeffs* co,
                                                const double* d_f, const double* d_g, const ihdg_options* opts,
                                                double* d_u, double* d_tr, void* stream, ihdg_result* res) {
  if (!ctx) return IHDG_ERR_INVALID;
  if (!mesh || !co || !d_f || !d_g || !d_u) return fail(ctx, IHDG_ERR_INVALID, "null argument");
  if (co->pde == IHDG_SWE) return fail(ctx, IHDG_ERR_INVALID, "shallow water is solved by ihdg_swe_steps*");
  ihdg_options o = defaults(opts);
  ihdg_status st = check_opts(ctx, o);
  if (st != IHDG_OK) return st;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const auto t_setup = std::chrono::steady_clock::now();
  Plan pl;
  st = prepare_plan(ctx, *mesh, *co, pl);
  if (st != IHDG_OK) return st;
  const Layout L = layout_for(pl.g, o, false);
  const size_t need = align256(pl.dbytes) + L.total;
  if (need > (size_t)IHDG_STATIC_SCRATCH_BYTES) {
    std::ostringstream os;
    os << "problem needs " << need << " bytes of scratch; ihdg_solve_device_static holds at most "
       << (size_t)IHDG_STATIC_SCRATCH_BYTES << " (use ihdg_solve_device with a caller workspace)";
    return fail(ctx, IHDG_ERR_NOMEM, os.str());
  }
  void* base = nullptr;
  st = static_scratch(ctx, &base);
  if (st != IHDG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = upload_plan(ctx, pl, base, s);
  if (st != IHDG_OK) return st;
  // this path builds and uploads the operators on every call (nothing is cached)
  const double setup_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_setup).count();
  SrcDev src{d_f, d_g, nullptr};
  st = device_iterate(ctx, &pl, o, src, o.u0, d_u, d_tr, static_cast<char*>(base) + align256(pl.dbytes), L, s, res);
  if (st != IHDG_OK) return st;
  if (res) res->setup_ms = setup_ms;
  ctx->err.clear();
  return IHDG_OK;
}

// ---------------------------------------------------------------------------------------
// Serving: continuous batching of independent solve requests.
//
// The server owns one device arena of the HBM budget.  ihdg_submit validates and copies a
// request, prepares its operators on the caller's thread, and queues it.  Each of the
// server's slots is a host thread with its own context (pinned loop-state readback), its own
// CUDA stream and one request at a time: it takes the first queued request whose footprint
// (operator image + workspace + inputs + outputs) fits in the arena's free space, runs the
// solve on its stream, copies the results back and frees its space, then takes the next.
// Requests that arrive while others run are admitted as soon as a slot and memory free up,
// and the slots' kernels overlap on the device.  A request's launch configuration depends
// only on its own size, so its result is the same alone and in any mix.
namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  long long id = 0;
  Plan plan;
  ihdg_options opts{};
  std::vector<double> f, g, u, tr;
  size_t fbytes = 0, gbytes = 0, ubytes = 0, tbytes = 0, footprint = 0, arena_off = 0;
  Layout L{};
  ihdg_result res{};
  ihdg_status st = IHDG_OK;
  std::string err;
  int state = 0;   // 0 queued, 1 running, 2 done
  double t_submit = 0, t_start = 0, t_end = 0;
};

struct Server {
  int device = 0;
  char* arena = nullptr;
  size_t budget = 0;
  std::vector<std::pair<size_t, size_t>> free_list;   // (offset, size), sorted by offset
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::unordered_map<long long, std::unique_ptr<Request>> all;
  std::vector<std::thread> workers;
  std::vector<ihdg_ctx*> slot_ctx;
  std::vector<cudaStream_t> streams;
  bool stop = false;
  long long next_id = 1;

  bool alloc(size_t bytes, size_t* off) {   // first fit; caller holds mu
    for (size_t i = 0; i < free_list.size(); ++i) {
      if (free_list[i].second >= bytes) {
        *off = free_list[i].first;
        free_list[i].first += bytes;
        free_list[i].second -= bytes;
        if (free_list[i].second == 0) free_list.erase(free_list.begin() + i);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {   // caller holds mu; coalesce neighbours
    auto it = free_list.begin();
    while (it != free_list.end() && it->first < off) ++it;
    it = free_list.insert(it, {off, bytes});
    if (it + 1 != free_list.end() && it->first + it->second == (it + 1)->first) {
      it->second += (it + 1)->second;
      free_list.erase(it + 1);
    }
    if (it != free_list.begin() && (it - 1)->first + (it - 1)->second == it->first) {
      (it - 1)->second += it->second;
      free_list.erase(it);
    }
  }
};

void serve_one(ihdg_ctx* sctx, cudaStream_t stream, Server* sv, Request* r) {
  char* base = sv->arena + r->arena_off;
  double* d_f = reinterpret_cast<double*>(base);
  double* d_g = reinterpret_cast<double*>(base + r->fbytes);
  double* d_u = reinterpret_cast<double*>(base + r->fbytes + r->gbytes);
  double* d_t = reinterpret_cast<double*>(base + r->fbytes + r->gbytes + r->ubytes);
  char* img = base + r->fbytes + r->gbytes + r->ubytes + r->tbytes;
  char* ws = img + align256(r->plan.dbytes);
  ihdg_status st = IHDG_OK;
  cudaError_t e = cudaMemcpyAsync(d_f, r->f.data(), r->f.size() * sizeof(double), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_g, r->g.data(), r->g.size() * sizeof(double), cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) { st = IHDG_ERR_CUDA; sctx->err = cudaGetErrorString(e); }
  if (st == IHDG_OK) st = upload_plan(sctx, r->plan, img, stream);
  if (st == IHDG_OK) {
    SrcDev src{d_f, d_g, nullptr};
    st = device_iterate(sctx, &r->plan, r->opts, src, nullptr, d_u, d_t, ws, r->L, stream, &r->res);
  }
  if (st == IHDG_OK) {
    e = cudaMemcpyAsync(r->u.data(), d_u, r->u.size() * sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->tr.data(), d_t, r->tr.size() * sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) { st = IHDG_ERR_CUDA; sctx->err = cudaGetErrorString(e); }
  }
  // the request's space goes back to the arena after this returns: drain the stream on
  // every path (an error may leave kernels or copies queued that still write to it)
  cudaStreamSynchronize(stream);
  r->st = st;
  if (st != IHDG_OK) r->err = sctx->err;
}

void slot_loop(Server* sv, int slot) {
  cudaSetDevice(sv->device);
  ihdg_ctx* sctx = sv->slot_ctx[slot];
  cudaStream_t stream = sv->streams[slot];
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      for (;;) {
        if (sv->stop) return;
        for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
          size_t off = 0;
          if (sv->alloc((*it)->footprint, &off)) {
            r = *it;
            r->arena_off = off;
            r->state = 1;
            r->t_start = now_ms();
            sv->queue.erase(it);
            break;
          }
        }
        if (r) break;
        sv->cv.wait(lk);
      }
    }
    serve_one(sctx, stream, sv, r);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->release(r->arena_off, r->footprint);
      r->t_end = now_ms();
      r->res.latency_ms = r->t_end - r->t_submit;
      r->res.queue_ms = r->t_start - r->t_submit;
      r->state = 2;
    }
    sv->cv.notify_all();
  }
}

}  // namespace

extern "C" ihdg_status ihdg_server_start(ihdg_ctx* ctx, size_t hbm_budget_bytes, int slots) {
  if (!ctx) return IHDG_ERR_INVALID;
  if (ctx->server) return fail(ctx, IHDG_ERR_INVALID, "the server is already running");
  if (slots < 1 || slots > 64) return fail(ctx, IHDG_ERR_INVALID, "slots must be in 1..64");
  if (hbm_budget_bytes < (1u << 20)) return fail(ctx, IHDG_ERR_INVALID, "hbm_budget_bytes must be at least 1 MiB");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  auto sv = std::make_unique<Server>();
  sv->device = ctx->device;
  sv->budget = hbm_budget_bytes & ~size_t(255);
  cudaError_t e = cudaMalloc(&sv->arena, sv->budget);
  if (e != cudaSuccess) return fail(ctx, IHDG_ERR_NOMEM, std::string("server arena: ") + cudaGetErrorString(e));
  sv->free_list.push_back({0, sv->budget});
  for (int i = 0; i < slots; ++i) {
    ihdg_ctx* c = nullptr;
    cudaStream_t s = nullptr;
    if (ihdg_create(&c, ctx->device) != IHDG_OK || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto* x : sv->slot_ctx) ihdg_destroy(x);
      for (auto x : sv->streams) cudaStreamDestroy(x);
      if (c) ihdg_destroy(c);
      cudaFree(sv->arena);
      return fail(ctx, IHDG_ERR_CUDA, "server slot set-up failed");
    }
    sv->slot_ctx.push_back(c);
    sv->streams.push_back(s);
  }
  Server* raw = sv.release();
  for (int i = 0; i < slots; ++i) raw->workers.emplace_back(slot_loop, raw, i);
  ctx->server = raw;
  ctx->err.clear();
  return IHDG_OK;
}

extern "C" ihdg_status ihdg_server_stop(ihdg_ctx* ctx) {
  if (!ctx) return IHDG_ERR_INVALID;
  Server* sv = ctx->server;
  if (!sv) return IHDG_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (auto& t : sv->workers) t.join();   // a running request finishes first
  cudaSetDevice(sv->device);
  for (auto* c : sv->slot_ctx) ihdg_destroy(c);
  for (auto s : sv->streams) cudaStreamDestroy(s);
  cudaFree(sv->arena);
  delete sv;
  ctx->server = nullptr;
  return IHDG_OK;
}

extern "C" ihdg_status ihdg_submit(ihdg_ctx* ctx, const ihdg_mesh* mesh, const ihdg_coeffs* co, const double* f_qp,
                                   const double* g_qp, const ihdg_options* opts, ihdg_ticket* out) {
  if (!ctx) return IHDG_ERR_INVALID;
  Server* sv = ctx->server;
  if (!sv) return fail(ctx, IHDG_ERR_INVALID, "no server: call ihdg_server_start first");
  if (!mesh || !co || !f_qp || !g_qp || !out) return fail(ctx, IHDG_ERR_INVALID, "null argument");
  if (co->pde == IHDG_SWE) return fail(ctx, IHDG_ERR_INVALID, "shallow water is solved by ihdg_swe_steps*");
  auto r = std::make_unique<Request>();
  r->t_submit = now_ms();
  r->opts = defaults(opts);
  r->opts.u0 = nullptr;
  r->opts.profile = 0;
  ihdg_status st = check_opts(ctx, r->opts);
  if (st != IHDG_OK) return st;
  if (r->opts.krylov_restart > 0)
    return fail(ctx, IHDG_ERR_UNSUPPORTED, "served requests run Algorithm 1 (opts.krylov_restart = 0)");
  st = prepare_plan(ctx, *mesh, *co, r->plan);
  if (st != IHDG_OK) return st;
  ihdg_sizes sz;
  ihdg_problem_sizes(mesh, co, &sz);
  r->f.assign(f_qp, f_qp + (size_t)sz.n_el * sz.nqv);
  r->g.assign(g_qp, g_qp + (size_t)sz.n_bface * sz.nqf);
  r->u.resize((size_t)sz.n_el * sz.nvol);
  r->tr.resize((size_t)sz.n_face * sz.nface_nodes);
  r->fbytes = align256(r->f.size() * sizeof(double));
  r->gbytes = align256(r->g.size() * sizeof(double));
  r->ubytes = align256(r->u.size() * sizeof(double));
  r->tbytes = align256(r->tr.size() * sizeof(double));
  r->L = layout_for(r->plan.g, r->opts, false);
  r->footprint = r->fbytes + r->gbytes + r->ubytes + r->tbytes + align256(r->plan.dbytes) + r->L.total;
  if (r->footprint > sv->budget) {
    std::ostringstream os;
    os << "request needs " << r->footprint << " bytes of HBM, the server budget is " << sv->budget;
    return fail(ctx, IHDG_ERR_NOMEM, os.str());
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->id = sv->next_id++;
    *out = r->id;
    sv->queue.push_back(r.get());
    sv->all.emplace(r->id, std::move(r));
  }
  sv->cv.notify_all();
  ctx->err.clear();
  return IHDG_OK;
}

extern "C" ihdg_status ihdg_poll(ihdg_ctx* ctx, ihdg_ticket t, ihdg_result* res) {
  if (!ctx) return IHDG_ERR_INVALID;
  Server* sv = ctx->server;
  if (!sv) return fail(ctx, IHDG_ERR_INVALID, "no server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(t);
  if (it == sv->all.end()) return fail(ctx, IHDG_ERR_INVALID, "unknown ticket");
  Request* r = it->second.get();
  if (r->state != 2) return IHDG_ERR_BUSY;
  if (r->st != IHDG_OK) return fail(ctx, r->st, r->err);
  if (res) *res = r->res;
  return IHDG_OK;
}

extern "C" ihdg_status ihdg_fetch(ihdg_ctx* ctx, ihdg_ticket t, double* u_out, double* trace_out) {
  if (!ctx) return IHDG_ERR_INVALID;
  Server* sv = ctx->server;
  if (!sv) return fail(ctx, IHDG_ERR_INVALID, "no server");
  std::unique_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(t);
    if (it == sv->all.end()) return fail(ctx, IHDG_ERR_INVALID, "unknown ticket");
    if (it->second->state != 2) return IHDG_ERR_BUSY;
    r = std::move(it->second);
    sv->all.erase(it);
  }
  if (r->st != IHDG_OK) return fail(ctx, r->st, r->err);
  if (u_out) std::memcpy(u_out, r->u.data(), r->u.size() * sizeof(double));
  if (trace_out) std::memcpy(trace_out, r->tr.data(), r->tr.size() * sizeof(double));
  return IHDG_OK;
}

ihdg_status ihdg_swe_steps_device(ihdg_ctx* ctx, const ihdg_mesh* mesh, const ihdg_coeffs* co, double* d_q,
                                  int nsteps, const ihdg_options* opts, int* iters_per_step, void* d_ws,
                                  size_t ws_bytes, void* stream, ihdg_result* res) {
  if (!ctx) return IHDG_ERR_INVALID;
  if (!mesh || !co || !d_q || !d_ws) return fail(ctx, IHDG_ERR_INVALID, "null argument");
  if (co->pde != IHDG_SWE) return fail(ctx, IHDG_ERR_INVALID, "ihdg_swe_steps* needs coeffs.pde = IHDG_SWE");
  if (nsteps < 0) return fail(ctx, IHDG_ERR_INVALID, "nsteps must be >= 0");
  if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0) return fail(ctx, IHDG_ERR_INVALID, "workspace must be 256-byte aligned");
  ihdg_options o = defaults(opts);
  ihdg_status st = check_opts(ctx, o);
  if (st != IHDG_OK) return st;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  // Crank-Nicolson: the backward-Euler half step (operators at dt/2) to tolerance tol/2, then
  // q^{m+1} = 2 q^{m+1/2} - q^m (see ihdg_time_scheme)
  // Automatic inner cap of the warm-started steps: 32 inner sweeps per outer step.  Their
  // inner loops stall above ~1e-2 of ||r|| (the inner stopping ratio is then never met), so
  // the general cap of 400 spends sweeps without progress; measured on 512^2 p=2, 100 steps,
  // mixed float32: 99.6 -> 33.2 sweeps per step, 271 -> 197 ms (cap 12: 201 ms, 64: 203 ms).
  if (!opts || opts->inner_max <= 0) o.inner_max = 32;
  const bool cn = co->time_scheme == IHDG_CRANK_NICOLSON;
  ihdg_coeffs cs = *co;
  if (cn) {
    cs.dt = 0.5 * co->dt;
    cs.time_scheme = IHDG_BACKWARD_EULER;
    o.tol = 0.5 * o.tol;
  }
  Plan* pl = nullptr;
  double setup_ms = 0.0;
  st = get_plan(ctx, *mesh, cs, pl, &setup_ms);
  if (st != IHDG_OK) return st;
  Layout L = layout_for(pl->g, o, true);
  if (ws_bytes < L.total) return fail(ctx, IHDG_ERR_NOMEM, "workspace smaller than ihdg_workspace_bytes()");
  char* ws = static_cast<char*>(d_ws);
  double* qn = reinterpret_cast<double*>(ws + L.qnext);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ihdg_result tot{};
  tot.status = IHDG_OK;
  size_t qbytes = sizeof(double) * (size_t)pl->g.nel * pl->g.nvol;
  for (int m = 0; m < nsteps; ++m) {
    SrcDev src{nullptr, nullptr, d_q};
    ihdg_result r{};
    st = device_iterate(ctx, pl, o, src, d_q, qn, nullptr, ws, L, s, &r);
    if (st != IHDG_OK) return st;
    if (cn) {
      CK(launch_cn_extrapolate(d_q, qn, (long long)pl->g.nel * pl->g.nvol, s), "Crank-Nicolson kernel");
      r.kernel_launches += 1;
      r.residual *= 2.0;   // the Crank-Nicolson iterate's increment
    } else {
      CK(cudaMemcpyAsync(d_q, qn, qbytes, cudaMemcpyDeviceToDevice, s), "copy q");
    }
    if (iters_per_step) iters_per_step[m] = r.iterations;
    tot.iterations += r.iterations;
    tot.fp64_sweeps += r.fp64_sweeps;
    tot.lowp_sweeps += r.lowp_sweeps;
    tot.solve_ms += r.solve_ms;
    tot.residual = r.residual;
    tot.fp64_sweep_ms += r.fp64_sweep_ms * r.fp64_launches;
    tot.lowp_sweep_ms += r.lowp_sweep_ms * r.lowp_launches;
    tot.fp64_launches += r.fp64_launches;
    tot.lowp_launches += r.lowp_launches;
    tot.kernel_launches += r.kernel_launches;
    if (r.inner_kernel_used) tot.inner_kernel_used = r.inner_kernel_used;
    if (r.status > tot.status) tot.status = r.status;
  }
  CK(cudaStreamSynchronize(s), "swe steps");
  if (tot.fp64_launches) tot.fp64_sweep_ms /= tot.fp64_launches;
  if (tot.lowp_launches) tot.lowp_sweep_ms /= tot.lowp_launches;
  tot.setup_ms = setup_ms;
  if (res) *res = tot;
  ctx->err.clear();
  return IHDG_OK;
}

ihdg_status ihdg_swe_steps(ihdg_ctx* ctx, const ihdg_mesh* mesh, const ihdg_coeffs* co, double* q, int nsteps,
                           const ihdg_options* opts, int* iters_per_step, ihdg_result* res) {
  if (!ctx) return IHDG_ERR_INVALID;
  if (!mesh || !co || !q) return fail(ctx, IHDG_ERR_INVALID, "null argument");
  ihdg_sizes sz;
  ihdg_status st = ihdg_problem_sizes(mesh, co, &sz);
  if (st != IHDG_OK) {
    std::string err;
    validate(*mesh, co, err);
    return fail(ctx, st, err.empty() ? "invalid problem" : err);
  }
  ihdg_options o = defaults(opts);
  size_t ws = 0;
  ihdg_workspace_bytes(mesh, co, &o, &ws);
  size_t bq = align256(sizeof(double) * sz.n_el * sz.nvol);
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  st = ensure_scratch(ctx, bq + ws);
  if (st != IHDG_OK) return st;
  double* d_q = static_cast<double*>(ctx->scratch);
  CK(cudaMemcpy(d_q, q, sizeof(double) * sz.n_el * sz.nvol, cudaMemcpyHostToDevice), "copy q");
  st = ihdg_swe_steps_device(ctx, mesh, co, d_q, nsteps, &o, iters_per_step, static_cast<char*>(ctx->scratch) + bq, ws, nullptr, res);
  if (st != IHDG_OK) return st;
  CK(cudaMemcpy(q, d_q, sizeof(double) * sz.n_el * sz.nvol, cudaMemcpyDeviceToHost), "copy q");
  return IHDG_OK;
}

// ---------------------------------------------------------------------------------------
// Transport with a velocity field that varies in space: plans of per-element local solves.

// ---------------------------------------------------------------------------------------
// Grouped float64 solves: every problem's init kernels, then one cooperative launch per
// element shape for the problems whose blocks fit together (each problem's loop exactly as
// in its own launch), then the rest one by one, then every reconstruction; one readback.
ihdg_status ihdg_group_workspace_bytes(int n, const ihdg_mesh* meshes, const ihdg_coeffs* coeffs,
                                       const ihdg_options* opts, size_t* bytes) {
  if (n < 0 || !bytes || (n > 0 && (!meshes || !coeffs))) return IHDG_ERR_INVALID;
  size_t tot = sweep64_group_desc_bytes(n);
  for (int i = 0; i < n; ++i) {
    if (coeffs[i].pde == IHDG_SWE) return IHDG_ERR_INVALID;
    size_t b = 0;
    ihdg_status st = ihdg_workspace_bytes(&meshes[i], &coeffs[i], opts, &b);
    if (st != IHDG_OK) return st;
    tot += align256(b);
  }
  *bytes = tot;
  return IHDG_OK;
}

ihdg_status ihdg_solve_group_device(ihdg_ctx* ctx, int n, const ihdg_mesh* meshes, const ihdg_coeffs* coeffs,
                                    const double* const* d_f, const double* const* d_g, const ihdg_options* opts,
                                    double* const* d_u, double* const* d_tr, void* d_ws, size_t ws_bytes,
                                    void* stream, ihdg_result* res) {
  if (!ctx) return IHDG_ERR_INVALID;
  if (n < 0) return fail(ctx, IHDG_ERR_INVALID, "n must be >= 0");
  if (n == 0) return IHDG_OK;
  if (!meshes || !coeffs || !d_f || !d_g || !d_u || !d_ws) return fail(ctx, IHDG_ERR_INVALID, "null argument");
  if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0) return fail(ctx, IHDG_ERR_INVALID, "workspace must be 256-byte aligned");
  ihdg_options o = defaults(opts);
  ihdg_status st = check_opts(ctx, o);
  if (st != IHDG_OK) return st;
  if (o.prec != IHDG_FP64) return fail(ctx, IHDG_ERR_UNSUPPORTED, "grouped solves run the float64 path (opts.prec = IHDG_FP64)");
  if (o.krylov_restart > 0)
    return fail(ctx, IHDG_ERR_UNSUPPORTED, "grouped solves run Algorithm 1 (opts.krylov_restart = 0)");
  if (o.u0) return fail(ctx, IHDG_ERR_UNSUPPORTED, "grouped solves start from the zero guess (opts.u0 = NULL)");
  size_t need = 0;
  st = ihdg_group_workspace_bytes(n, meshes, coeffs, &o, &need);
  if (st != IHDG_OK) return fail(ctx, st, "invalid problem in the group");
  if (ws_bytes < need) return fail(ctx, IHDG_ERR_NOMEM, "workspace smaller than ihdg_group_workspace_bytes()");
  for (int i = 0; i < n; ++i)
    if (!d_f[i] || !d_g[i] || !d_u[i]) return fail(ctx, IHDG_ERR_INVALID, "null argument");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the plans stay in the context's cache for the whole call
  struct Pin {
    ihdg_ctx* c;
    ~Pin() { c->plan_pin -= 1; }
  } pin{ctx};
  ctx->plan_pin += 1;
  // the failure-detection hooks of the single solve (a block that never arrives, a shorter
  // bound of every wait), read the same way
  long long wait_cycles = 2000000000LL;
  int stall_block = -1;
  if (const char* w = std::getenv("IHDG_TEST_WAIT_CYCLES")) {
    const long long v = std::atoll(w);
    if (v > 0) wait_cycles = v;
  }
  if (const char* b = std::getenv("IHDG_TEST_STALL_BLOCK")) stall_block = std::atoi(b);
  std::vector<Plan*> pl((size_t)n, nullptr);
  std::vector<double> setup((size_t)n, 0.0);
  std::vector<LaunchArgs> a((size_t)n);
  std::vector<Layout> L((size_t)n);
  char* ws = static_cast<char*>(d_ws);
  char* desc = ws;
  size_t at = sweep64_group_desc_bytes(n);
  for (int i = 0; i < n; ++i) {
    st = get_plan(ctx, meshes[i], coeffs[i], pl[(size_t)i], &setup[(size_t)i]);
    if (st != IHDG_OK) return st;
    L[(size_t)i] = layout_for(pl[(size_t)i]->g, o, false);
    char* w = ws + at;
    at += align256(L[(size_t)i].total);
    LaunchArgs& ai = a[(size_t)i];
    ai = LaunchArgs{};
    ai.g = pl[(size_t)i]->g;
    ai.op = pl[(size_t)i]->op;
    ai.src = SrcDev{d_f[i], d_g[i], nullptr};
    ai.u0 = nullptr;
    ai.F = reinterpret_cast<double*>(w + L[(size_t)i].F);
    ai.V = reinterpret_cast<double*>(w + L[(size_t)i].V);
    ai.ring = reinterpret_cast<double*>(w + L[(size_t)i].ring);
    ai.ring_stride = (long long)ai.g.n_exp * ai.g.ld;
    ai.ctrl = reinterpret_cast<Ctrl*>(w + L[(size_t)i].ctrl);
    ai.partials = reinterpret_cast<double*>(w + L[(size_t)i].partials);
    ai.res_hist = reinterpret_cast<double*>(w + L[(size_t)i].res_hist);
    ai.stream = s;
    CK(launch_ctrl_init(ai, o.tol, o.diverge_factor, o.max_iters, o.inner_max, o.inner_rtol, wait_cycles, stall_block),
       "ctrl init");
    CK(launch_forcing(ai), "forcing kernel");
    CK(launch_export0(ai, nullptr, ai.ring), "initial export kernel");
    CK(launch_first(ai), "first sweep kernel");
  }
  // one cooperative launch per element shape, as many problems as fit together (in order)
  std::vector<int> rest;
  std::vector<char> placed((size_t)n, 0);
  for (int i = 0; i < n; ++i) {
    if (placed[(size_t)i]) continue;
    std::vector<LaunchArgs> cls;
    std::vector<int> idx;
    for (int j = i; j < n; ++j)
      if (!placed[(size_t)j] && a[(size_t)j].g.dim == a[(size_t)i].g.dim && a[(size_t)j].g.nf == a[(size_t)i].g.nf) {
        cls.push_back(a[(size_t)j]);
        idx.push_back(j);
        placed[(size_t)j] = 1;
      }
    size_t k = 0;
    while (k < cls.size()) {
      // the largest prefix of the remaining problems that is co-resident
      size_t m = cls.size() - k;
      cudaError_t e = cudaErrorNotSupported;
      while (m > 0) {
        e = launch_sweep64_persist_group(cls.data() + k, (int)m, desc, s);
        if (e != cudaErrorNotSupported) break;
        cudaGetLastError();
        m = m > 1 ? m / 2 : 0;
      }
      if (e != cudaSuccess && e != cudaErrorNotSupported) return cuda_fail(ctx, e, "grouped sweep kernel");
      if (m == 0) {   // too large for a persistent launch: its own loop below
        rest.push_back(idx[k]);
        k += 1;
        continue;
      }
      // (the next launch's descriptor copy is stream-ordered after this launch)
      k += m;
    }
  }
  std::vector<Ctrl> hc((size_t)n);
  for (int i : rest) {   // batches of launches with host checks, as the single solve does
    LaunchArgs& ai = a[(size_t)i];
    int batch = 2;
    for (;;) {
      CK(cudaMemcpyAsync(&hc[(size_t)i], ai.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s), "ctrl readback");
      CK(cudaStreamSynchronize(s), "sweep loop");
      if (hc[(size_t)i].done) break;
      int left = hc[(size_t)i].max_iters - hc[(size_t)i].iter;
      int nb = batch < left ? batch : left;
      if (nb <= 0) break;
      CK(launch_sweep64(ai, nb), "sweep kernel");
      if (batch < 32) batch *= 2;
    }
  }
  for (int i = 0; i < n; ++i)
    CK(cudaMemcpyAsync(&hc[(size_t)i], a[(size_t)i].ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s), "ctrl readback");
  CK(cudaStreamSynchronize(s), "grouped solves");
  for (int i = 0; i < n; ++i) {
    const LaunchArgs& ai = a[(size_t)i];
    if (hc[(size_t)i].timeout) return fail(ctx, IHDG_ERR_TIMEOUT, "grouped float64 sweep: a grid barrier wait ran out");
    const int K = hc[(size_t)i].iter;
    const double* Et = ai.ring + (long long)(K % 3) * ai.ring_stride;
    const double* Eu = ai.ring + (long long)((K + 2) % 3) * ai.ring_stride;
    CK(launch_reconstruct(ai, Eu, nullptr, d_u[i]), "reconstruct kernel");
    if (d_tr && d_tr[i]) {
      const Plan* p = pl[(size_t)i];
      double beta[3] = {p->co.beta[0], p->co.beta[1], p->co.beta[2]};
      CK(launch_trace_out(ai, Et, nullptr, d_u[i], (int)p->co.pde, beta, p->ops.alpha_axis, count_faces(p->mesh, nullptr),
                          d_tr[i]),
         "trace kernel");
    }
    if (res) {
      ihdg_result r{};
      r.iterations = hc[(size_t)i].iter;
      r.fp64_sweeps = hc[(size_t)i].fp64_sweeps;
      r.residual = hc[(size_t)i].res;
      r.status = (ihdg_status)hc[(size_t)i].status;
      r.setup_ms = setup[(size_t)i];
      res[i] = r;
    }
  }
  CK(cudaStreamSynchronize(s), "grouped reconstructions");
  ctx->err.clear();
  return IHDG_OK;
}

}  // extern "C"

struct ihdg_var_plan {
  int device = 0;
  ihdg_mesh mesh{};
  ihdg::VarDev dev;
  long long n_el = 0, n_bface = 0, n_face = 0;
  int nvol = 0, nqv = 0, nqf = 0, nf = 0;
  double setup_ms = 0.0;
};

extern "C" {

ihdg_status ihdg_face_quadrature_points(const ihdg_mesh* mesh, double* xyz) {
  if (!mesh || !xyz) return IHDG_ERR_INVALID;
  std::string err;
  ihdg_status st = validate(*mesh, nullptr, err);
  if (st != IHDG_OK) return st;
  face_points(*mesh, xyz);
  return IHDG_OK;
}

ihdg_status ihdg_var_plan_create(ihdg_ctx* ctx, const ihdg_mesh* mesh, const double* beta_vol, const double* beta_face,
                                 ihdg_var_plan** out) {
  if (!ctx) return IHDG_ERR_INVALID;
  if (!mesh || !beta_vol || !beta_face || !out) return fail(ctx, IHDG_ERR_INVALID, "null argument");
  *out = nullptr;
  const auto t0 = std::chrono::steady_clock::now();
  VarHost h;
  std::string err;
  ihdg_status st = build_var(*mesh, beta_vol, beta_face, h, err);
  if (st != IHDG_OK) return fail(ctx, st, err);
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  auto pl = std::make_unique<ihdg_var_plan>();
  pl->device = ctx->device;
  pl->mesh = *mesh;
  cudaError_t e = var_upload(h, pl->dev, 100000);
  if (e != cudaSuccess) {
    const ihdg_status code = e == cudaErrorMemoryAllocation ? IHDG_ERR_NOMEM : IHDG_ERR_CUDA;
    return fail(ctx, code, std::string("variable-coefficient plan upload: ") + cudaGetErrorString(e));
  }
  pl->n_el = h.nel;
  pl->n_bface = h.nbface;
  pl->n_face = h.nface;
  pl->nvol = h.nb;
  pl->nqv = h.nqv;
  pl->nqf = h.nqf;
  pl->nf = h.nf;
  pl->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = pl.release();
  ctx->err.clear();
  return IHDG_OK;
}

void ihdg_var_plan_destroy(ihdg_var_plan* plan) {
  if (!plan) return;
  cudaSetDevice(plan->device);
  var_free(plan->dev);
  delete plan;
}

ihdg_status ihdg_var_plan_info(const ihdg_var_plan* plan, size_t* device_bytes, double* setup_ms) {
  if (!plan) return IHDG_ERR_INVALID;
  if (device_bytes) *device_bytes = plan->dev.bytes;
  if (setup_ms) *setup_ms = plan->setup_ms;
  return IHDG_OK;
}

ihdg_status ihdg_var_host_operator(const ihdg_mesh* mesh, const double* beta_vol, const double* beta_face,
                                   long long element, int which, int* rows, int* cols, double* data) {
  if (!mesh || !beta_vol || !beta_face || !rows || !cols) return IHDG_ERR_INVALID;
  VarHost h;
  std::string err;
  ihdg_status st = build_var(*mesh, beta_vol, beta_face, h, err);
  if (st != IHDG_OK) return st;
  if (element < 0 || element >= h.nel || (which != 0 && which != 1)) return IHDG_ERR_INVALID;
  *rows = h.nb;
  *cols = which == 0 ? h.nin : h.nb;
  if (!data) return IHDG_OK;
  const int nc = *cols;
  const double* src = which == 0 ? &h.L[(size_t)element * h.nin * h.nb] : &h.Ainv[(size_t)element * h.nb * h.nb];
  for (int i = 0; i < h.nb; ++i)
    for (int k = 0; k < nc; ++k) data[(size_t)i * nc + k] = src[(size_t)k * h.nb + i];   // stored column by column
  return IHDG_OK;
}

ihdg_status ihdg_var_solve_device(ihdg_ctx* ctx, ihdg_var_plan* plan, const double* d_f, const double* d_g,
                                  const ihdg_options* opts, double* d_u, double* d_tr, void* stream, ihdg_result* res) {
  if (!ctx) return IHDG_ERR_INVALID;
  if (!plan || !d_f || !d_g || !d_u) return fail(ctx, IHDG_ERR_INVALID, "null argument");
  if (plan->device != ctx->device) return fail(ctx, IHDG_ERR_INVALID, "the plan belongs to another device");
  ihdg_options o = defaults(opts);
  ihdg_status st = check_opts(ctx, o);
  if (st != IHDG_OK) return st;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  std::string err;
  st = var_solve(plan->dev, d_f, d_g, o, d_u, d_tr, static_cast<cudaStream_t>(stream), ctx->h_ctrl, err, res);
  if (st != IHDG_OK) return fail(ctx, st, err);
  ctx->err.clear();
  return IHDG_OK;
}

ihdg_status ihdg_var_solve_group(ihdg_ctx* ctx, int n, ihdg_var_plan* const* plans, const double* const* d_f,
                                 const double* const* d_g, const ihdg_options* opts, double* const* d_u,
                                 double* const* d_tr, void* stream, ihdg_result* res) {
  if (!ctx) return IHDG_ERR_INVALID;
  if (n < 1 || n > 64) return fail(ctx, IHDG_ERR_INVALID, "n must be in 1..64");
  if (!plans || !d_f || !d_g || !d_u || !res) return fail(ctx, IHDG_ERR_INVALID, "null argument");
  ihdg_options o = defaults(opts);
  ihdg_status st = check_opts(ctx, o);
  if (st != IHDG_OK) return st;
  if (o.u0) return fail(ctx, IHDG_ERR_INVALID, "a grouped solve takes no initial guess (opts->u0 must be NULL)");
  std::vector<VarDev*> ds;
  std::vector<const double*> fv, gv;
  std::vector<double*> uv, tv;
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !d_f[i] || !d_g[i] || !d_u[i]) return fail(ctx, IHDG_ERR_INVALID, "null argument");
    if (plans[i]->device != ctx->device) return fail(ctx, IHDG_ERR_INVALID, "a plan belongs to another device");
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return fail(ctx, IHDG_ERR_INVALID, "a plan appears twice in the group");
    ds.push_back(&plans[i]->dev);
    fv.push_back(d_f[i]);
    gv.push_back(d_g[i]);
    uv.push_back(d_u[i]);
    tv.push_back(d_tr ? d_tr[i] : nullptr);
  }
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  std::string err;
  st = var_solve_group(ds, fv, gv, o, uv, tv, static_cast<cudaStream_t>(stream), err, res);
  if (st != IHDG_OK) return fail(ctx, st, err);
  ctx->err.clear();
  return IHDG_OK;
}

ihdg_status ihdg_var_solve(ihdg_ctx* ctx, ihdg_var_plan* plan, const double* f_qp, const double* g_qp,
                           const ihdg_options* opts, double* u_out, double* trace_out, ihdg_result* res) {
  if (!ctx) return IHDG_ERR_INVALID;
  if (!plan || !f_qp || !g_qp || !u_out) return fail(ctx, IHDG_ERR_INVALID, "null argument");
  if (plan->device != ctx->device) return fail(ctx, IHDG_ERR_INVALID, "the plan belongs to another device");
  ihdg_options o = defaults(opts);
  ihdg_status st = check_opts(ctx, o);
  if (st != IHDG_OK) return st;
  const size_t bf = align256(sizeof(double) * plan->n_el * plan->nqv), bg = align256(sizeof(double) * plan->n_bface * plan->nqf);
  const size_t bu = align256(sizeof(double) * plan->n_el * plan->nvol), bt = align256(sizeof(double) * plan->n_face * plan->nf);
  const size_t bu0 = o.u0 ? bu : 0;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  st = ensure_scratch(ctx, bf + bg + bu + bt + bu0);
  if (st != IHDG_OK) return st;
  char* s = static_cast<char*>(ctx->scratch);
  double* d_f = reinterpret_cast<double*>(s);
  double* d_g = reinterpret_cast<double*>(s + bf);
  double* d_u = reinterpret_cast<double*>(s + bf + bg);
  double* d_t = reinterpret_cast<double*>(s + bf + bg + bu);
  double* d_u0 = o.u0 ? reinterpret_cast<double*>(s + bf + bg + bu + bt) : nullptr;
  CK(cudaMemcpy(d_f, f_qp, sizeof(double) * plan->n_el * plan->nqv, cudaMemcpyHostToDevice), "copy f");
  CK(cudaMemcpy(d_g, g_qp, sizeof(double) * plan->n_bface * plan->nqf, cudaMemcpyHostToDevice), "copy g");
  if (o.u0) CK(cudaMemcpy(d_u0, o.u0, sizeof(double) * plan->n_el * plan->nvol, cudaMemcpyHostToDevice), "copy u0");
  ihdg_options od = o;
  od.u0 = d_u0;
  st = ihdg_var_solve_device(ctx, plan, d_f, d_g, &od, d_u, trace_out ? d_t : nullptr, nullptr, res);
  if (st != IHDG_OK) return st;
  CK(cudaMemcpy(u_out, d_u, sizeof(double) * plan->n_el * plan->nvol, cudaMemcpyDeviceToHost), "copy u");
  if (trace_out) CK(cudaMemcpy(trace_out, d_t, sizeof(double) * plan->n_face * plan->nf, cudaMemcpyDeviceToHost), "copy trace");
  return IHDG_OK;
}

// Host-only inspection of the float64 operators of a problem (no device needed).
// which: 0 L_E, 1 Q, 2 L_vol, 3 R, 4 PF, 5 PV.  rows/cols receive the shape; data may be
// NULL to query the shape only.
ihdg_status ihdg_host_operator(const ihdg_mesh* mesh, const ihdg_coeffs* co, int which, int* rows, int* cols,
                               double* data) {
  if (!mesh || !co || !rows || !cols) return IHDG_ERR_INVALID;
  std::string err;
  Ops o;
  ihdg_status st = build_ops(*mesh, *co, o, err);
  if (st != IHDG_OK) return st;
  const std::vector<double>* v = nullptr;
  int r = 0, c = 0;
  switch (which) {
    case 0: v = &o.LE; r = o.n_exp; c = o.n_in; break;
    case 1: v = &o.Q; r = o.n_in; c = o.n_in; break;
    case 2: v = &o.Lvol; r = o.nvol; c = o.n_in; break;
    case 3: v = &o.R; r = o.n_exp; c = o.nvol; break;
    case 4: v = &o.PF; r = o.n_exp; c = o.nqv; break;
    case 5: v = &o.PV; r = o.nvol; c = o.nqv; break;
    default: return IHDG_ERR_INVALID;
  }
  *rows = r;
  *cols = c;
  if (data && v->size() == (size_t)r * c) std::memcpy(data, v->data(), sizeof(double) * v->size());
  return IHDG_OK;
}

}  // extern "C"
