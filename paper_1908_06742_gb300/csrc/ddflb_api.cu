// C ABI of the DDF lattice Boltzmann library (declared in include/ddflb.h).
//
// Host-side runtime: parameter validation, workspace carving (the caller owns
// all device memory), the step loop with its periodic reductions, host-staged
// I/O, checkpoints and thread-local error messages.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "../../include/ddflb.h"
#include "ddflb_internal.h"

using namespace ddflb;

namespace {

thread_local std::string g_err;

ddflb_status fail(ddflb_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

ddflb_status cuda_fail(cudaError_t e, const char* where) {
  return fail(DDFLB_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

constexpr size_t kAlign = 256;
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t elem_size(int storage) { return storage == DDFLB_FP32 ? 4 : 2; }

struct Layout {
  int pitch;
  int ghost_lo, ghost_hi;  // 1 where a y-slab shares its bottom / top face with another slab
  int buf_ny;              // rows of the population buffers: own rows + ghost rows
  size_t gofs;             // bytes from a buffer's flow planes to its scalar planes
  size_t pops_bytes;  // one buffer: 2 lattices x 9 planes
  size_t off_a, off_b, off_uprev, off_part, off_status, off_stage, off_stage_out, total;
};

// Row pitch: a multiple of 64 elements keeps every row start 128-byte aligned
// for 16-bit storage and 256-byte aligned for FP32.  p->ny is the number of
// rows the context owns (the whole lattice, or one y-slab).
Layout layout(const ddflb_params* p, int ghost_lo = 0, int ghost_hi = 0) {
  Layout L{};
  L.pitch = (int)align_up((size_t)p->nx, 64);
  L.ghost_lo = ghost_lo;
  L.ghost_hi = ghost_hi;
  L.buf_ny = p->ny + ghost_lo + ghost_hi;
  const size_t plane = (size_t)L.pitch * L.buf_ny;
  const size_t cells = (size_t)p->nx * p->ny;
  L.gofs = 9 * plane * elem_size(p->storage);
  L.pops_bytes = align_up(2 * 9 * plane * elem_size(p->storage), kAlign);
  size_t o = 0;
  L.off_a = o; o += L.pops_bytes;
  L.off_b = o; o += L.pops_bytes;
  L.off_uprev = o; o += align_up(2 * cells * sizeof(float), kAlign);
  L.off_part = o; o += align_up((size_t)kReduceBlocks * 4 * sizeof(double), kAlign);
  L.off_status = o; o += align_up(sizeof(DevStatus), kAlign);
  L.off_stage = o;  // host I/O: 10 input planes, then 8 output planes
  if (p->flags & DDFLB_FLAG_HOST_IO) o += align_up(10 * cells * sizeof(float), kAlign);
  L.off_stage_out = o;
  if (p->flags & DDFLB_FLAG_HOST_IO) o += align_up(8 * cells * sizeof(float), kAlign);
  L.total = o;
  return L;
}

ddflb_status validate(const ddflb_params* p) {
  if (!p) return fail(DDFLB_EINVAL, "params is NULL");
  if (p->bc < 0 || p->bc > 2) return fail(DDFLB_EINVAL, "bc %d is not a ddflb_bc", p->bc);
  const int minx = p->bc == DDFLB_BC_CHANNEL ? 1 : 2;
  if (p->nx < minx || p->ny < 2) return fail(DDFLB_EINVAL, "grid %d x %d too small", p->nx, p->ny);
  // a population plane (rows padded to 64 nodes) is indexed with 32-bit offsets
  if (((int64_t)p->nx + 63) / 64 * 64 * p->ny >= (int64_t)1 << 32)
    return fail(DDFLB_EINVAL, "grid %d x %d: a padded plane reaches 2^32 nodes", p->nx, p->ny);
  if (p->storage < 0 || p->storage > 2) return fail(DDFLB_EINVAL, "storage %d invalid", p->storage);
  for (int k = 0; k < 9; ++k) {
    if (!(p->omega_f[k] >= 0.0 && p->omega_f[k] <= 2.0))
      return fail(DDFLB_EINVAL, "omega_f[%d] = %g outside [0, 2]", k, p->omega_f[k]);
    if (!(p->omega_g[k] >= 0.0 && p->omega_g[k] <= 2.0))
      return fail(DDFLB_EINVAL, "omega_g[%d] = %g outside [0, 2]", k, p->omega_g[k]);
  }
  if (p->omega_f[0] != 0 || p->omega_f[1] != 0 || p->omega_f[2] != 0)
    return fail(DDFLB_EINVAL, "omega_f[0..2] must be 0 (mass and momentum are conserved)");
  if (p->omega_g[0] != 0) return fail(DDFLB_EINVAL, "omega_g[0] must be 0 (phi is conserved)");
  if (!(std::fabs(p->beta1 - p->beta2) > 1e-6))
    return fail(DDFLB_EINVAL, "beta1 - beta2 = %g: the vorticity needs beta1 != beta2",
                p->beta1 - p->beta2);
  if (std::fabs(p->cs2 - 1.0 / 3.0) > 1e-12 || std::fabs(p->cs2_phi - 1.0 / 3.0) > 1e-12)
    return fail(DDFLB_EINVAL, "cs2 and cs2_phi must be 1/3 (the D2Q9 rest weights)");
  if (!std::isfinite(p->rho0) || p->rho0 <= 0) return fail(DDFLB_EINVAL, "rho0 must be > 0");
  if (!std::isfinite(p->phi0) || !std::isfinite(p->u_lid) || !std::isfinite(p->phi_lid) ||
      !std::isfinite(p->phi_wall) || !(p->phi_min >= 0))
    return fail(DDFLB_EINVAL, "non-finite boundary or reference value");
  if (p->check_every < 0) return fail(DDFLB_EINVAL, "check_every < 0");
  if (!std::isfinite(p->fx) || !std::isfinite(p->fy) || !std::isfinite(p->force_omega))
    return fail(DDFLB_EINVAL, "non-finite body force or force frequency");
  if (p->scalar_model < 0 || p->scalar_model > 3)
    return fail(DDFLB_EINVAL, "scalar_model %d is not a ddflb_scalar_model", p->scalar_model);
  if (p->reserved != 0) return fail(DDFLB_EINVAL, "reserved must be 0");
  for (double s : {p->scale_f, p->scale_g}) {
    if (s > 0) {
      int e;
      if (std::frexp(s, &e) != 0.5) return fail(DDFLB_EINVAL, "scale %g is not a power of two", s);
    }
  }
  return DDFLB_OK;
}

LbParams make_lb(const ddflb_params* p, int pitch, int ghost_lo = 0, int ghost_hi = 0) {
  LbParams P{};
  P.nx = p->nx;
  P.ny = p->ny + ghost_lo + ghost_hi;
  P.y0 = ghost_lo;
  P.y1 = ghost_lo + p->ny;
  P.pitch = pitch;
  P.plane = (int64_t)pitch * P.ny;
  for (int k = 0; k < 9; ++k) {
    P.wf[k] = (float)p->omega_f[k];
    // SRT (App. B): one rate for every non-conserved scalar moment
    const double wg = p->scalar_model == DDFLB_SCALAR_SRT && k > 0 ? p->omega_g[1] : p->omega_g[k];
    P.wg[k] = (float)wg;
  }
  P.smodel = p->scalar_model;
  P.b1 = (float)p->beta1;
  P.b2 = (float)p->beta2;
  P.inv_db = (float)(1.0 / (p->beta1 - p->beta2));
  P.cs2 = (float)p->cs2;
  P.cs2p = (float)p->cs2_phi;
  P.rho0 = (float)p->rho0;
  P.phi0 = (float)p->phi0;
  P.phimin = (float)p->phi_min;
  const bool half = p->storage != DDFLB_FP32;
  const double sf = half && p->scale_f > 0 ? p->scale_f : 1.0;
  const double sg = half && p->scale_g > 0 ? p->scale_g : 1.0;
  P.sf = (float)sf;
  P.isf = (float)(1.0 / sf);
  P.sg = (float)sg;
  P.isg = (float)(1.0 / sg);
  // rest weights from the equilibrium at u = 0 through the inverse of App. B:
  // w0 = (1 - c)^2, w1..4 = c (1 - c) / 2, w5..8 = c^2 / 4
  auto weights = [](double c, float* w) {
    w[0] = (float)((1 - c) * (1 - c));
    for (int a = 1; a <= 4; ++a) w[a] = (float)(c * (1 - c) / 2);
    for (int a = 5; a <= 8; ++a) w[a] = (float)(c * c / 4);
  };
  weights(p->cs2, P.wrf);
  weights(p->cs2_phi, P.wrg);
  static const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  for (int a = 0; a < 9; ++a) {
    const double wf = P.wrf[a], wg = P.wrg[a];
    P.lid[a] = (float)(2.0 * wf * p->rho0 * ex[a] * p->u_lid / p->cs2);
    P.abb_lid[a] = (float)(2.0 * wg * (p->phi_lid - p->phi0));
    P.abb_wall[a] = (float)(2.0 * wg * (p->phi_wall - p->phi0));
  }
  P.fx = (float)p->fx;
  P.fy = (float)p->fy;
  P.fmod = 1.0f;
  P.ffield = nullptr;
  return P;
}

}  // namespace

namespace ddflb {
void set_error(const char* msg) { g_err = msg; }
LbParams make_lbparams(const ddflb_params* p, int pitch) { return make_lb(p, pitch); }
}  // namespace ddflb

struct ddflb_ctx {
  ddflb_params p;
  Layout lay;
  Launch L;
  char* ws;
  void* pops[2];
  int cur;  // pops[cur] holds the current (post-collision, pre-stream) state
  float* uprev;
  double* partials;
  DevStatus* status;
  float* stage;
  int64_t step;
  int64_t snap_step;  // step at which uprev was last written (-1: none)
  int path;           // step kernel: 0 default (16-bit storage: groups of 4 nodes, else
                      // pairs on a periodic lattice, where eligible; else one node),
                      // 1 one node per thread, 2 paired nodes, 3 groups of 4 nodes
  float* stage_out;   // output staging area (host I/O)
  cudaStream_t io_up, io_down;  // streams of host uploads / downloads (null: the context stream)
  cudaEvent_t ev_in_free, ev_in_ready, ev_out_ready, ev_out_free;  // host-I/O ordering
  // kGraphSteps steps captured as one CUDA graph, starting from pops[0] / pops[1]
  // (null: not built yet); graph_failed: capture unavailable, launch step by step
  cudaGraphExec_t step_graph[2];
  bool graph_failed;
  int32_t slab_y0;    // first global row of a y-slab context (0 for a whole lattice)
  int32_t global_ny;  // rows of the whole lattice
};

namespace {
// NVTX range over one host call (visible in profilers; a no-op without one)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// Body-force modulation cos(force_omega t) for the launches that act on the
// state at time t (the collision of step t, and fields / sums of state t).
void at_time(ddflb_ctx* c, int64_t t) {
  c->L.P.fmod = c->p.force_omega != 0.0 ? (float)std::cos(c->p.force_omega * (double)t) : 1.0f;
}

bool has_force(const ddflb_params& p, const float* field) {
  return p.fx != 0.0 || p.fy != 0.0 || field != nullptr;
}
}  // namespace

namespace ddflb {
// 16-bit storage, two adjacent nodes per thread (ddflb_step_pair.cu)
bool pair_step_eligible(const Launch& L);
cudaError_t launch_step_pair(const Launch& L, const void* fin, const void* gin, void* fout,
                             void* gout, const DevStatus* st);
// periodic 16-bit lattices with nx a multiple of 4: four nodes per thread
bool quad_step_eligible(const Launch& L);
cudaError_t launch_step_quad(const Launch& L, const void* fin, const void* gin, void* fout,
                             void* gout, const DevStatus* st);
}  // namespace ddflb

namespace {
cudaError_t run_step(const ddflb_ctx* c, const void* fin, const void* gin, void* fout, void* gout) {
  // 16-bit storage steps node groups by default (wider accesses; bit-identical)
  if ((c->path == 3 || c->path == 0) && quad_step_eligible(c->L))
    return launch_step_quad(c->L, fin, gin, fout, gout, c->status);
  // (with walls the paired kernel is no faster than one node per thread)
  const bool pair = c->path == 2 || c->path == 3 ||
                    (c->path == 0 && c->L.storage != 0 && c->L.P_bc == BC_PERIODIC);
  if (pair && pair_step_eligible(c->L))
    return launch_step_pair(c->L, fin, gin, fout, gout, c->status);
  return launch_step(c->L, fin, gin, fout, gout, c->status);
}

// Small lattices are launch-bound: runs of kGraphSteps steps between checks
// replay one captured graph (an even count, so the buffer parity returns).
// Only without a time-modulated force (whose factor changes every step).
constexpr int kGraphSteps = 64;

void drop_graphs(ddflb_ctx* c) {
  for (cudaGraphExec_t& g : c->step_graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

// The graph of kGraphSteps steps that starts from pops[c->cur], built on first
// use (null if capture is unavailable: the caller then launches step by step).
cudaGraphExec_t step_graph(ddflb_ctx* c) {
  const int p = c->cur;
  if (c->step_graph[p] || c->graph_failed) return c->step_graph[p];
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->graph_failed = true;
    return nullptr;
  }
  const cudaStream_t saved = c->L.stream;
  c->L.stream = cs;
  cudaGraph_t g = nullptr;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  for (int i = 0, cur = p; ok && i < kGraphSteps; ++i, cur ^= 1) {
    char* fo = (char*)c->pops[cur ^ 1];
    const size_t gofs = c->lay.gofs;
    ok = run_step(c, c->pops[cur], (const char*)c->pops[cur] + gofs, fo, fo + gofs) ==
         cudaSuccess;
  }
  if (cudaStreamEndCapture(cs, &g) != cudaSuccess) ok = false;
  c->L.stream = saved;
  cudaGraphExec_t ex = nullptr;
  if (ok && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ok = false;
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  cudaGetLastError();  // clear a capture error, if any
  if (!ok) {
    c->graph_failed = true;
    return nullptr;
  }
  c->step_graph[p] = ex;
  return ex;
}
}  // namespace

namespace {

const void* fptr(const ddflb_ctx* c, int buf) { return c->pops[buf]; }

// Zero the device status block (no residual yet, not diverged) on the stream.
ddflb_status reset_status(ddflb_ctx* c) {
  cudaError_t e = cudaMemsetAsync(c->status, 0, sizeof(DevStatus), c->L.stream);
  return e == cudaSuccess ? DDFLB_OK : cuda_fail(e, "status reset");
}

const void* gptr(const ddflb_ctx* c, int buf) { return (const char*)c->pops[buf] + c->lay.gofs; }

ddflb_status check_launch(cudaError_t e, const char* where) {
  return e == cudaSuccess ? DDFLB_OK : cuda_fail(e, where);
}

ddflb_status reduce(ddflb_ctx* c, int mode) {
  at_time(c, c->step);
  cudaError_t e = launch_reduce(c->L, fptr(c, c->cur), gptr(c, c->cur), c->uprev, mode,
                                c->partials, c->status);
  if (e != cudaSuccess) return cuda_fail(e, "reduce");
  if (mode & 2) c->snap_step = c->step;
  return DDFLB_OK;
}

// Residual bookkeeping at state time s: at every multiple of K the velocity is
// compared with the snapshot taken K steps earlier, then becomes the next
// snapshot (one pass).  The reported residual is |u(s) - u(s-K)| / (K |u(s)|).
ddflb_status checks_at(ddflb_ctx* c) {
  const int K = c->p.check_every;
  if (K <= 0) return DDFLB_OK;
  const int64_t s = c->step;
  if (s % K != 0) return DDFLB_OK;
  const int mode = (s > 0 && c->snap_step == s - K ? 1 : 0) | 2;
  return reduce(c, mode);
}

}  // namespace

extern "C" {

size_t ddflb_workspace_bytes(const ddflb_params* p) {
  if (validate(p) != DDFLB_OK) return 0;
  return layout(p).total;
}

}  // extern "C"

namespace {
// Geometry of a y-slab [y0, y0 + rows) of the lattice *p: the slab's own
// parameters (ny = rows) and its ghost rows (one on each face shared with
// another slab: both faces of a periodic lattice's slab, the inner faces of a
// walled one).
ddflb_status slab_geometry(const ddflb_params* p, int32_t y0, int32_t rows, ddflb_params* own,
                           int* glo, int* ghi) {
  ddflb_status s = validate(p);
  if (s != DDFLB_OK) return s;
  if (y0 < 0 || rows < 1 || (int64_t)y0 + rows > p->ny)
    return fail(DDFLB_EINVAL, "slab rows [%d, %lld) outside 0..%d", y0, (long long)y0 + rows, p->ny);
  *own = *p;
  own->ny = rows;
  const bool whole = rows == p->ny;
  if (p->bc == DDFLB_BC_PERIODIC) {
    *glo = *ghi = whole ? 0 : 1;
  } else {
    *glo = y0 > 0 ? 1 : 0;
    *ghi = y0 + rows < p->ny ? 1 : 0;
  }
  if ((*glo || *ghi) && p->check_every != 0)
    return fail(DDFLB_EINVAL, "a y-slab context reduces through ddflb_sums: check_every must be 0");
  if ((*glo || *ghi) && p->force_omega != 0.0)
    return fail(DDFLB_EINVAL, "y-slab contexts take steady forces only");
  if (((int64_t)p->nx + 63) / 64 * 64 * ((int64_t)rows + *glo + *ghi) >= (int64_t)1 << 32)
    return fail(DDFLB_EINVAL, "slab of %d x %d: a padded plane reaches 2^32 nodes", p->nx, rows);
  return DDFLB_OK;
}

ddflb_status create_ctx(const ddflb_params* p, int glo, int ghi, int32_t y0, int32_t global_ny,
                        void* ws, size_t bytes, void* stream, ddflb_ctx** out) {
  if (!ws) return fail(DDFLB_EINVAL, "workspace is NULL");
  if ((uintptr_t)ws % kAlign) return fail(DDFLB_EINVAL, "workspace not %zu-byte aligned", kAlign);
  const Layout lay = layout(p, glo, ghi);
  if (bytes < lay.total)
    return fail(DDFLB_ENOMEM, "workspace %zu bytes < %zu required", bytes, lay.total);
  ddflb_ctx* c = new (std::nothrow) ddflb_ctx();
  if (!c) return fail(DDFLB_ENOMEM, "host allocation of the handle failed");
  c->p = *p;
  c->lay = lay;
  c->slab_y0 = y0;
  c->global_ny = global_ny;
  c->ws = (char*)ws;
  c->pops[0] = c->ws + lay.off_a;
  c->pops[1] = c->ws + lay.off_b;
  c->cur = 0;
  c->uprev = (float*)(c->ws + lay.off_uprev);
  c->partials = (double*)(c->ws + lay.off_part);
  c->status = (DevStatus*)(c->ws + lay.off_status);
  c->stage = (p->flags & DDFLB_FLAG_HOST_IO) ? (float*)(c->ws + lay.off_stage) : nullptr;
  c->stage_out = (p->flags & DDFLB_FLAG_HOST_IO) ? (float*)(c->ws + lay.off_stage_out) : nullptr;
  c->L.P = make_lb(p, lay.pitch, glo, ghi);
  c->L.P_bc = p->bc;
  c->L.storage = p->storage;
  c->L.force = has_force(*p, nullptr);
  c->L.block = dim3(128, 1, 1);
  c->L.stream = (cudaStream_t)stream;
  c->step = 0;
  c->snap_step = -1;
  ddflb_status st = reset_status(c);
  if (st != DDFLB_OK) {
    delete c;
    return st;
  }
  *out = c;
  return DDFLB_OK;
}
}  // namespace

extern "C" {

ddflb_status ddflb_create(const ddflb_params* p, void* ws, size_t bytes, void* stream,
                          ddflb_ctx** out) {
  if (!out) return fail(DDFLB_EINVAL, "out is NULL");
  *out = nullptr;
  ddflb_status s = validate(p);
  if (s != DDFLB_OK) return s;
  return create_ctx(p, 0, 0, 0, p->ny, ws, bytes, stream, out);
}

size_t ddflb_slab_workspace_bytes(const ddflb_params* p, int32_t y0, int32_t rows) {
  ddflb_params own;
  int glo = 0, ghi = 0;
  if (slab_geometry(p, y0, rows, &own, &glo, &ghi) != DDFLB_OK) return 0;
  return layout(&own, glo, ghi).total;
}

ddflb_status ddflb_slab_create(const ddflb_params* p, int32_t y0, int32_t rows, void* ws,
                               size_t bytes, void* stream, ddflb_ctx** out) {
  if (!out) return fail(DDFLB_EINVAL, "out is NULL");
  *out = nullptr;
  ddflb_params own;
  int glo = 0, ghi = 0;
  ddflb_status s = slab_geometry(p, y0, rows, &own, &glo, &ghi);
  if (s != DDFLB_OK) return s;
  return create_ctx(&own, glo, ghi, y0, p->ny, ws, bytes, stream, out);
}

ddflb_status ddflb_init(ddflb_ctx* c, const float* rho, const float* ux, const float* uy,
                        const float* phi, const float* grads) {
  if (!c || !rho || !ux || !uy || !phi) return fail(DDFLB_EINVAL, "NULL handle or field");
  Range range("ddflb_init");
  if (grads) {
    const double* wf = c->p.omega_f;
    const float* wg = c->L.P.wg;
    if (wf[3] <= 0 || wf[4] <= 0 || wf[5] <= 0 || wg[1] <= 0 || wg[2] <= 0 || wg[5] <= 0)
      return fail(DDFLB_EINVAL, "gradient initialisation needs w3, w4, w5, w1^phi, w2^phi, "
                                "w5^phi > 0");
  }
  ddflb_status s = reset_status(c);
  if (s != DDFLB_OK) return s;
  c->cur = 0;
  c->step = 0;
  c->snap_step = -1;
  at_time(c, 0);
  InitPtrs in{rho, ux, uy, phi, grads};
  void* f = c->pops[0];
  void* g = (char*)f + c->lay.gofs;
  s = check_launch(launch_init(c->L, in, f, g), "init");
  if (s != DDFLB_OK) return s;
  return checks_at(c);
}

// Host-I/O ordering between a copy stream and the compute stream (no-op when
// the copies run on the compute stream itself).
static cudaError_t io_order(bool separate, cudaStream_t waiter, cudaEvent_t ev,
                            cudaStream_t recorder) {
  if (!separate) return cudaSuccess;
  cudaError_t e = cudaEventRecord(ev, recorder);
  return e == cudaSuccess ? cudaStreamWaitEvent(waiter, ev, 0) : e;
}

ddflb_status ddflb_init_host(ddflb_ctx* c, const float* rho, const float* ux, const float* uy,
                             const float* phi, const float* grads) {
  if (!c || !rho || !ux || !uy || !phi) return fail(DDFLB_EINVAL, "NULL handle or field");
  if (!c->stage) return fail(DDFLB_EINVAL, "context created without DDFLB_FLAG_HOST_IO");
  const size_t n = (size_t)c->p.nx * c->p.ny;
  const float* src[5] = {rho, ux, uy, phi, grads};
  const size_t planes[5] = {1, 1, 1, 1, 6};
  float* dst[5];
  const bool sep = c->io_up != nullptr;
  cudaStream_t cs = sep ? c->io_up : c->L.stream;
  // the upload waits until the previous init has read the staging area
  cudaError_t e = sep ? cudaStreamWaitEvent(cs, c->ev_in_free, 0) : cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(e, "init_host order");
  size_t o = 0;
  for (int k = 0; k < 5; ++k) {
    dst[k] = c->stage + o * n;
    o += planes[k];
    if (!src[k]) continue;
    e = cudaMemcpyAsync(dst[k], src[k], planes[k] * n * sizeof(float), cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "init_host copy");
  }
  e = io_order(sep, c->L.stream, c->ev_in_ready, cs);
  if (e != cudaSuccess) return cuda_fail(e, "init_host order");
  ddflb_status s = ddflb_init(c, dst[0], dst[1], dst[2], dst[3], grads ? dst[4] : nullptr);
  if (s != DDFLB_OK) return s;
  e = sep ? cudaEventRecord(c->ev_in_free, c->L.stream) : cudaSuccess;
  return e == cudaSuccess ? DDFLB_OK : cuda_fail(e, "init_host order");
}

ddflb_status ddflb_step(ddflb_ctx* c, int64_t n) {
  if (!c) return fail(DDFLB_EINVAL, "NULL handle");
  if (n < 0) return fail(DDFLB_EINVAL, "n < 0");
  if (n > 1 && (c->lay.ghost_lo || c->lay.ghost_hi))
    return fail(DDFLB_EINVAL, "a y-slab context takes one step per call: its ghost rows are "
                              "refreshed between steps");
  Range range("ddflb_step");
  const int K = c->p.check_every;
  while (n > 0) {
    if (c->p.force_omega == 0.0 && !c->graph_failed) {
      // whole graphs up to the next check step (checks run after it, as below)
      const int64_t until = K > 0 ? std::min<int64_t>(n, K - c->step % K) : n;
      const int64_t reps = until / kGraphSteps;
      at_time(c, c->step);  // (the factor is 1 at every step here)
      cudaGraphExec_t ex = reps > 0 ? step_graph(c) : nullptr;
      if (ex) {
        Range graphs("ddflb_step graph replay");
        for (int64_t r = 0; r < reps; ++r) {
          cudaError_t e = cudaGraphLaunch(ex, c->L.stream);
          if (e != cudaSuccess) return cuda_fail(e, "step graph");
        }
        c->step += reps * kGraphSteps;
        n -= reps * kGraphSteps;
        ddflb_status s = checks_at(c);
        if (s != DDFLB_OK) return s;
        continue;
      }
    }
    --n;
    const int src = c->cur, dst = c->cur ^ 1;
    void* fo = c->pops[dst];
    void* go = (char*)fo + c->lay.gofs;
    at_time(c, c->step);
    cudaError_t e = run_step(c, fptr(c, src), gptr(c, src), fo, go);
    if (e != cudaSuccess) return cuda_fail(e, "step");
    c->cur = dst;
    ++c->step;
    ddflb_status s = checks_at(c);
    if (s != DDFLB_OK) return s;
  }
  return DDFLB_OK;
}

ddflb_status ddflb_fields(ddflb_ctx* c, float* rho, float* ux, float* uy, float* phi, float* sxx,
                          float* sxy, float* syy, float* omega) {
  if (!c) return fail(DDFLB_EINVAL, "NULL handle");
  Range range("ddflb_fields");
  FieldPtrs fp{{rho, ux, uy, phi, sxx, sxy, syy, omega}};
  at_time(c, c->step);
  return check_launch(launch_fields(c->L, fptr(c, c->cur), gptr(c, c->cur), fp), "fields");
}

ddflb_status ddflb_derived(ddflb_ctx* c, float* dxux, float* dyux, float* dxuy, float* dyuy,
                           float* dxphi, float* dyphi, float* q, float* r, float* lamb_x,
                           float* lamb_y) {
  if (!c) return fail(DDFLB_EINVAL, "NULL handle");
  FieldPtrs fp{};
  float* d[10] = {dxux, dyux, dxuy, dyuy, dxphi, dyphi, q, r, lamb_x, lamb_y};
  for (int k = 0; k < 10; ++k) fp.p[8 + k] = d[k];
  fp.derived = 1;
  at_time(c, c->step);
  return check_launch(launch_fields(c->L, fptr(c, c->cur), gptr(c, c->cur), fp), "derived");
}

ddflb_status ddflb_fields_host_async(ddflb_ctx* c, float* rho, float* ux, float* uy, float* phi,
                                     float* sxx, float* sxy, float* syy, float* omega) {
  if (!c) return fail(DDFLB_EINVAL, "NULL handle");
  if (!c->stage_out) return fail(DDFLB_EINVAL, "context created without DDFLB_FLAG_HOST_IO");
  const size_t n = (size_t)c->p.nx * c->p.ny;
  float* host[8] = {rho, ux, uy, phi, sxx, sxy, syy, omega};
  FieldPtrs fp{};
  for (int k = 0; k < 8; ++k) fp.p[k] = host[k] ? c->stage_out + k * n : nullptr;
  const bool sep = c->io_down != nullptr;
  cudaStream_t cs = sep ? c->io_down : c->L.stream;
  // the fields kernel waits until the previous download has drained the staging area
  cudaError_t e = sep ? cudaStreamWaitEvent(c->L.stream, c->ev_out_free, 0) : cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(e, "fields_host order");
  at_time(c, c->step);
  ddflb_status s =
      check_launch(launch_fields(c->L, fptr(c, c->cur), gptr(c, c->cur), fp), "fields_host");
  if (s != DDFLB_OK) return s;
  e = io_order(sep, cs, c->ev_out_ready, c->L.stream);
  if (e != cudaSuccess) return cuda_fail(e, "fields_host order");
  for (int k = 0; k < 8; ++k) {
    if (!host[k]) continue;
    e = cudaMemcpyAsync(host[k], fp.p[k], n * sizeof(float), cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) return cuda_fail(e, "fields_host copy");
  }
  e = sep ? cudaEventRecord(c->ev_out_free, cs) : cudaSuccess;
  return e == cudaSuccess ? DDFLB_OK : cuda_fail(e, "fields_host order");
}

ddflb_status ddflb_fields_host(ddflb_ctx* c, float* rho, float* ux, float* uy, float* phi,
                               float* sxx, float* sxy, float* syy, float* omega) {
  ddflb_status s = ddflb_fields_host_async(c, rho, ux, uy, phi, sxx, sxy, syy, omega);
  return s == DDFLB_OK ? ddflb_io_wait(c) : s;
}

ddflb_status ddflb_io_wait(ddflb_ctx* c) {
  if (!c) return fail(DDFLB_EINVAL, "NULL handle");
  cudaError_t e = cudaStreamSynchronize(c->io_up ? c->io_up : c->L.stream);
  if (e == cudaSuccess && c->io_down) e = cudaStreamSynchronize(c->io_down);
  return e == cudaSuccess ? DDFLB_OK : cuda_fail(e, "io_wait");
}

ddflb_status ddflb_set_io_streams(ddflb_ctx* c, void* upload_stream, void* download_stream) {
  if (!c) return fail(DDFLB_EINVAL, "NULL handle");
  if (!c->stage) return fail(DDFLB_EINVAL, "context created without DDFLB_FLAG_HOST_IO");
  if ((upload_stream == nullptr) != (download_stream == nullptr) ||
      (upload_stream && upload_stream == download_stream))
    return fail(DDFLB_EINVAL, "give two distinct I/O streams, or none");
  if (upload_stream && !c->ev_in_free) {
    cudaEvent_t* evs[4] = {&c->ev_in_free, &c->ev_in_ready, &c->ev_out_ready, &c->ev_out_free};
    for (cudaEvent_t* ev : evs) {
      cudaError_t e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(e, "io events");
    }
  }
  // copies queued so far complete before the streams change roles
  ddflb_status s = ddflb_io_wait(c);
  if (s != DDFLB_OK) return s;
  c->io_up = (cudaStream_t)upload_stream;
  c->io_down = (cudaStream_t)download_stream;
  return DDFLB_OK;
}

ddflb_status ddflb_populations(ddflb_ctx* c, float* f, float* g) {
  if (!c) return fail(DDFLB_EINVAL, "NULL handle");
  return check_launch(launch_pops(c->L, fptr(c, c->cur), gptr(c, c->cur), f, g), "populations");
}

ddflb_status ddflb_stats(ddflb_ctx* c, double* mass, double* scalar, double* residual,
                         int64_t* step) {
  if (!c) return fail(DDFLB_EINVAL, "NULL handle");
  ddflb_status s = reduce(c, 0);
  if (s != DDFLB_OK) return s;
  DevStatus h{};
  cudaError_t e = cudaMemcpyAsync(&h, c->status, sizeof h, cudaMemcpyDeviceToHost, c->L.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->L.stream);
  if (e != cudaSuccess) return cuda_fail(e, "stats");
  const double cells = (double)c->p.nx * c->p.ny;
  if (mass) *mass = cells * c->p.rho0 + h.mass_dev;
  if (scalar) *scalar = cells * c->p.phi0 + h.scalar_dev;
  if (residual) *residual = h.has_residual ? h.residual / c->p.check_every : NAN;
  if (step) *step = c->step;
  if (h.diverged) return fail(DDFLB_EDIVERGED, "non-finite mass/scalar sum by step %lld",
                              (long long)c->step);
  return DDFLB_OK;
}

// Run to steady state (Sec. 5.4 reports the cavity flows at steady state):
// steps in chunks up to each check and reads the residual the check left in
// the status block.
ddflb_status ddflb_run_to_tolerance(ddflb_ctx* c, double tol, int64_t max_steps,
                                    int32_t stall_checks, int64_t* steps_taken) {
  if (steps_taken) *steps_taken = 0;
  if (!c) return fail(DDFLB_EINVAL, "NULL handle");
  const int K = c->p.check_every;
  if (K <= 0) return fail(DDFLB_EINVAL, "run_to_tolerance needs check_every > 0");
  if (!(tol > 0.0) || max_steps < 0 || stall_checks < 0)
    return fail(DDFLB_EINVAL, "tol must be > 0, max_steps and stall_checks >= 0");
  Range range("ddflb_run_to_tolerance");
  double best = INFINITY;
  int since_best = 0;
  int64_t done = 0;
  while (done < max_steps) {
    const int64_t n = std::min<int64_t>(max_steps - done, K - c->step % K);
    ddflb_status s = ddflb_step(c, n);
    if (s != DDFLB_OK) return s;
    done += n;
    if (steps_taken) *steps_taken = done;
    if (c->step % K != 0) continue;  // the step limit ended the chunk before a check
    DevStatus h{};
    cudaError_t e = cudaMemcpyAsync(&h, c->status, sizeof h, cudaMemcpyDeviceToHost, c->L.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->L.stream);
    if (e != cudaSuccess) return cuda_fail(e, "run_to_tolerance");
    if (h.diverged)
      return fail(DDFLB_EDIVERGED, "non-finite mass/scalar sum by step %lld", (long long)c->step);
    if (!h.has_residual) continue;  // the first check only takes the snapshot
    const double r = h.residual / K;
    if (r < tol) return DDFLB_OK;
    if (r < best) {
      best = r;
      since_best = 0;
    } else if (stall_checks > 0 && ++since_best >= stall_checks) {
      return fail(DDFLB_ENOTCONVERGED,
                  "residual %.3g stalled: no check below its best %.3g for %d checks (step %lld)",
                  r, best, stall_checks, (long long)c->step);
    }
  }
  return fail(DDFLB_ENOTCONVERGED, "residual above %g after %lld steps", tol, (long long)done);
}

size_t ddflb_state_bytes(const ddflb_ctx* c) { return c ? c->lay.pops_bytes : 0; }

ddflb_status ddflb_get_state(ddflb_ctx* c, void* dst, size_t bytes, int64_t* step) {
  if (!c || !dst) return fail(DDFLB_EINVAL, "NULL argument");
  if (bytes < c->lay.pops_bytes) return fail(DDFLB_ENOMEM, "state buffer too small");
  cudaError_t e = cudaMemcpyAsync(dst, c->pops[c->cur], c->lay.pops_bytes,
                                  cudaMemcpyDeviceToDevice, c->L.stream);
  if (e != cudaSuccess) return cuda_fail(e, "get_state");
  if (step) *step = c->step;
  return DDFLB_OK;
}

ddflb_status ddflb_set_state(ddflb_ctx* c, const void* src, size_t bytes, int64_t step) {
  if (!c || !src) return fail(DDFLB_EINVAL, "NULL argument");
  if (bytes < c->lay.pops_bytes) return fail(DDFLB_ENOMEM, "state buffer too small");
  if (step < 0) return fail(DDFLB_EINVAL, "step < 0");
  cudaError_t e = cudaMemcpyAsync(c->pops[0], src, c->lay.pops_bytes, cudaMemcpyDeviceToDevice,
                                  c->L.stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_state");
  c->cur = 0;
  c->step = step;
  c->snap_step = -1;
  return reset_status(c);
}

ddflb_status ddflb_destroy(ddflb_ctx* c) {
  if (c) drop_graphs(c);
  if (c && c->ev_in_free) {
    cudaEvent_t evs[4] = {c->ev_in_free, c->ev_in_ready, c->ev_out_ready, c->ev_out_free};
    for (cudaEvent_t ev : evs)
      if (ev) cudaEventDestroy(ev);
  }
  delete c;
  return DDFLB_OK;
}

const char* ddflb_last_error(void) { return g_err.c_str(); }

const char* ddflb_version(void) { return "ddflb 0.1 (sm_103a)"; }

// Autotuner for the step kernel's block shape: each candidate runs trial_steps
// untimed, then trial_steps timed with CUDA events on the context stream; the
// fastest is kept.  The trials run on zeroed populations (the rest state), so
// the state is overwritten and the step counter reset: call before ddflb_init.
ddflb_status ddflb_autotune(ddflb_ctx* c, int32_t trial_steps, int32_t* block_x,
                            int32_t* block_y, int32_t* path, double* ms_per_step) {
  if (!c || trial_steps < 1) return fail(DDFLB_EINVAL, "NULL handle or trial_steps < 1");
  static const int shapes[][2] = {{128, 1}, {256, 1}, {64, 2}, {32, 4}, {64, 4}, {32, 8}, {64, 1}};
  cudaStream_t s = c->L.stream;
  cudaError_t e = cudaMemsetAsync(c->pops[0], 0, 2 * c->lay.pops_bytes, s);
  if (e != cudaSuccess) return cuda_fail(e, "autotune clear");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  dim3 bestb(128, 1, 1);
  int bestp = 1;
  const int saved_path = c->path;
  const size_t gofs = c->lay.gofs;
  for (int pth = 1; pth <= 3 && e == cudaSuccess; ++pth) {
    for (const auto& sh : shapes) {
      c->L.block = dim3(sh[0], sh[1], 1);
      c->path = pth;
      if (pth == 2 && !pair_step_eligible(c->L)) continue;
      // the 4-node kernel has its own 128 x 1 block: timed once
      if (pth == 3 && (!quad_step_eligible(c->L) || &sh != &shapes[0])) continue;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        if (rep == 1) e = cudaEventRecord(e0, s);
        for (int i = 0; i < trial_steps && e == cudaSuccess; ++i) {
          const int src = i & 1;
          char* fo = (char*)c->pops[src ^ 1];
          e = run_step(c, c->pops[src], (const char*)c->pops[src] + gofs, fo, fo + gofs);
        }
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) break;
      if (ms < best) {
        best = ms;
        bestb = c->L.block;
        bestp = pth;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->path = saved_path;
  if (e != cudaSuccess) return cuda_fail(e, "autotune trial");
  c->L.block = bestb;
  c->path = bestp;
  drop_graphs(c);
  if (path) *path = bestp;
  e = cudaMemsetAsync(c->pops[0], 0, 2 * c->lay.pops_bytes, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "autotune reset");
  c->cur = 0;
  c->step = 0;
  c->snap_step = -1;
  ddflb_status st = reset_status(c);
  if (st != DDFLB_OK) return st;
  if (block_x) *block_x = (int32_t)bestb.x;
  if (block_y) *block_y = (int32_t)bestb.y;
  if (ms_per_step) *ms_per_step = best / trial_steps;
  return DDFLB_OK;
}

ddflb_status ddflb_set_path(ddflb_ctx* c, int32_t path) {
  if (!c || path < 0 || path > 3) return fail(DDFLB_EINVAL, "path must be 0, 1, 2 or 3");
  c->path = path;
  drop_graphs(c);
  return DDFLB_OK;
}

ddflb_status ddflb_set_force_field(ddflb_ctx* c, const float* dev_field) {
  if (!c) return fail(DDFLB_EINVAL, "NULL handle");
  c->L.P.ffield = dev_field;
  c->L.force = has_force(c->p, dev_field);
  drop_graphs(c);
  return DDFLB_OK;
}

size_t ddflb_halo_elems(const ddflb_ctx* c) { return c ? 6 * (size_t)c->p.nx : 0; }

ddflb_status ddflb_halo_pack(ddflb_ctx* c, void* dev_down, void* dev_up) {
  if (!c) return fail(DDFLB_EINVAL, "NULL handle");
  if ((dev_down && !c->lay.ghost_lo) || (dev_up && !c->lay.ghost_hi))
    return fail(DDFLB_EINVAL, "halo_pack: a face without a neighbouring slab sends nothing");
  if (!dev_down && !dev_up) return DDFLB_OK;
  return check_launch(launch_halo_pack(c->L, c->pops[c->cur], c->lay.gofs, dev_down, dev_up),
                      "halo_pack");
}

ddflb_status ddflb_halo_unpack(ddflb_ctx* c, const void* dev_from_below,
                               const void* dev_from_above) {
  if (!c) return fail(DDFLB_EINVAL, "NULL handle");
  if ((dev_from_below && !c->lay.ghost_lo) || (dev_from_above && !c->lay.ghost_hi))
    return fail(DDFLB_EINVAL, "halo_unpack: a face without a neighbouring slab has no ghost row");
  if (!dev_from_below && !dev_from_above) return DDFLB_OK;
  return check_launch(launch_halo_unpack(c->L, c->pops[c->cur], c->lay.gofs, dev_from_below,
                                         dev_from_above),
                      "halo_unpack");
}

ddflb_status ddflb_halo_exchange_local(ddflb_ctx* const* slabs, int32_t parts) {
  if (!slabs || parts < 1) return fail(DDFLB_EINVAL, "no slabs");
  if (parts > kMaxLocalSlabs) return fail(DDFLB_EINVAL, "at most %d slabs", kMaxLocalSlabs);
  for (int k = 0; k < parts; ++k)
    if (!slabs[k]) return fail(DDFLB_EINVAL, "slab %d is NULL", k);
  const ddflb_ctx* a = slabs[0];
  if (parts == 1) {
    if (a->lay.ghost_lo || a->lay.ghost_hi)
      return fail(DDFLB_EINVAL, "one slab of a divided lattice has no neighbours to exchange with");
    return DDFLB_OK;  // a whole lattice: nothing crosses a face
  }
  HaloSlabs H{};
  H.n = parts;
  H.nx = a->p.nx;
  H.pitch = a->lay.pitch;
  H.periodic = a->p.bc == DDFLB_BC_PERIODIC;
  int32_t next_y0 = 0;
  for (int k = 0; k < parts; ++k) {
    const ddflb_ctx* c = slabs[k];
    if (c->p.nx != a->p.nx || c->p.storage != a->p.storage || c->p.bc != a->p.bc ||
        c->global_ny != a->global_ny || c->L.stream != a->L.stream || c->cur != a->cur)
      return fail(DDFLB_EINVAL, "slab %d is not a slab of the same lattice on the same stream, "
                                "at the same step", k);
    if (c->slab_y0 != next_y0)
      return fail(DDFLB_EINVAL, "slab %d starts at row %d, expected %d (give them bottom to top)",
                  k, c->slab_y0, next_y0);
    next_y0 += c->p.ny;
    // a face shared with a neighbour has a ghost row on both sides
    if (!c->lay.ghost_hi && k < parts - 1)
      return fail(DDFLB_EINVAL, "slab %d has no ghost row above", k);
    H.s[k] = HaloSlab{c->pops[c->cur], (int64_t)(c->lay.gofs / elem_size(c->p.storage)),
                      c->L.P.plane, c->L.P.y0, c->L.P.y1};
  }
  if (next_y0 != a->global_ny)
    return fail(DDFLB_EINVAL, "the slabs cover rows 0..%d of %d", next_y0, a->global_ny);
  return check_launch(launch_halo_local(H, a->p.storage, a->L.stream), "halo_exchange_local");
}

ddflb_status ddflb_sums(ddflb_ctx* c, int32_t mode, double* out) {
  if (!c || !out) return fail(DDFLB_EINVAL, "NULL argument");
  if (mode < 0 || mode > 3) return fail(DDFLB_EINVAL, "mode %d not in 0..3", mode);
  if ((mode & 1) && c->snap_step < 0)
    return fail(DDFLB_EINVAL, "no velocity snapshot stored (call with mode bit 2 first)");
  ddflb_status s = reduce(c, mode);
  if (s != DDFLB_OK) return s;
  DevStatus h{};
  cudaError_t e = cudaMemcpyAsync(&h, c->status, sizeof h, cudaMemcpyDeviceToHost, c->L.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->L.stream);
  if (e != cudaSuccess) return cuda_fail(e, "sums");
  out[0] = h.mass_dev;
  out[1] = h.scalar_dev;
  out[2] = h.u2;
  out[3] = (mode & 1) ? h.du2 : NAN;
  if (h.diverged) return fail(DDFLB_EDIVERGED, "non-finite sum by step %lld", (long long)c->step);
  return DDFLB_OK;
}

ddflb_status ddflb_set_block(ddflb_ctx* c, int32_t block_x, int32_t block_y) {
  if (!c) return fail(DDFLB_EINVAL, "NULL handle");
  if (block_x < 32 || block_y < 1 || block_x % 32 || block_x * block_y > 256 ||
      block_x * block_y < 32)
    return fail(DDFLB_EINVAL, "block %d x %d: x a multiple of 32, 32..256 threads", block_x,
                block_y);
  c->L.block = dim3(block_x, block_y, 1);
  drop_graphs(c);
  return DDFLB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Reductions without any device allocation (no counterpart in the paper).
//
// For callers that cannot allocate device memory at the point of the call: code
// paths where cudaMalloc is forbidden or unavailable (real-time loops, callbacks
// of a framework that owns all device memory, plug-ins handed only pre-existing
// buffers).  The scratch the reduction needs -- block partial sums, a status
// block and the velocity snapshot for the residual -- lives in one file-scope
// device array instead of a caller workspace.  Every GPU that loads this
// library holds that array (about 8.4 MB) until the process exits.
namespace {

struct NoallocScratch {
  double partials[kReduceBlocks * 4];
  DevStatus status;
  float uprev[2 * DDFLB_NOALLOC_MAX_NODES];
};

__device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
NoallocScratch* g_noalloc_addr[kMaxDevices];  // device address, per device ordinal
// grid of the stored velocity snapshot, per device ordinal ({0, 0}: none); the
// snapshot is indexed by node, so a residual needs the same nx and ny
int32_t g_noalloc_snapshot_grid[kMaxDevices][2];

// Forget the snapshot of device `dev` (caller holds g_noalloc_mutex).
void snap_clear(int dev) {
  g_noalloc_snapshot_grid[dev][0] = 0;
  g_noalloc_snapshot_grid[dev][1] = 0;
}

// Turns the status block into (mass, scalar, sum |u|^2, residual).
__global__ void k_noalloc_out(const DevStatus* st, double cells, double rho0, double phi0,
                              int mode, double* out) {
  if (threadIdx.x != 0) return;
  out[0] = cells * rho0 + st->mass_dev;
  out[1] = cells * phi0 + st->scalar_dev;
  out[2] = st->u2;
  out[3] = (mode & 1) ? st->residual : __longlong_as_double(0x7ff8000000000000LL);
}

}  // namespace

extern "C" ddflb_status ddflb_reduce_noalloc(const ddflb_params* p, const void* dev_state,
                                             size_t state_bytes, int32_t mode, double* dev_out,
                                             void* cuda_stream) {
  ddflb_status s = validate(p);
  if (s != DDFLB_OK) return s;
  if (!dev_state || !dev_out) return fail(DDFLB_EINVAL, "NULL state or output");
  if (mode < 0 || mode > 3) return fail(DDFLB_EINVAL, "mode %d not in 0..3", mode);
  if (p->fx != 0.0 || p->fy != 0.0 || p->force_omega != 0.0)
    return fail(DDFLB_EINVAL, "ddflb_reduce_noalloc takes unforced states only");
  const int64_t nodes = (int64_t)p->nx * p->ny;
  if (nodes > DDFLB_NOALLOC_MAX_NODES)
    return fail(DDFLB_EINVAL,
                "grid %d x %d has %lld nodes; ddflb_reduce_noalloc holds scratch for at most %d",
                p->nx, p->ny, (long long)nodes, DDFLB_NOALLOC_MAX_NODES);
  const Layout lay = layout(p);
  if (state_bytes < lay.pops_bytes)
    return fail(DDFLB_EINVAL, "state buffer %zu bytes < %zu", state_bytes, lay.pops_bytes);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(DDFLB_EINVAL, "device ordinal %d too large", dev);
  NoallocScratch* scratch = nullptr;
  {
    // First call on a device (with that device current): look up the address of
    // the scratch array.  That lookup is not capturable, so the first call on a
    // device must come before any stream capture.
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
      g_noalloc_addr[dev] = (NoallocScratch*)ptr;
    }
    scratch = g_noalloc_addr[dev];
    const int32_t* snap = g_noalloc_snapshot_grid[dev];
    if ((mode & 1) && (snap[0] != p->nx || snap[1] != p->ny))
      return fail(DDFLB_EINVAL, "no velocity snapshot of a %d x %d grid stored on device %d",
                  p->nx, p->ny, dev);
    // a snapshot about to be overwritten is no longer valid, whatever happens below
    if (mode & 2) snap_clear(dev);
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Launch L;
  L.P = make_lb(p, lay.pitch);
  L.P_bc = p->bc;
  L.storage = p->storage;
  L.force = false;
  L.block = dim3(128, 1, 1);
  L.stream = st;
  // the status block keeps the last call's contents: clear it (diverged flag, residual)
  e = cudaMemsetAsync(&scratch->status, 0, sizeof(DevStatus), st);
  if (e != cudaSuccess) return cuda_fail(e, "no-allocation status clear");
  const char* f = (const char*)dev_state;
  const char* g = f + lay.gofs;
  e = launch_reduce(L, f, g, scratch->uprev, mode, scratch->partials, &scratch->status);
  if (e != cudaSuccess) return cuda_fail(e, "no-allocation reduce");
  if (mode & 2) {
    // the snapshot counts as stored only once its writer was launched
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    g_noalloc_snapshot_grid[dev][0] = p->nx;
    g_noalloc_snapshot_grid[dev][1] = p->ny;
  }
  k_noalloc_out<<<1, 32, 0, st>>>(&scratch->status, (double)nodes, p->rho0, p->phi0, mode,
                                  dev_out);
  e = cudaGetLastError();
  return e == cudaSuccess ? DDFLB_OK : cuda_fail(e, "no-allocation output");
}
