// Batched persistent step: many independent lattice pairs of uneven sizes and
// parameters advance together in one cooperative launch per chunk of steps.
//
// Work list: every instance is cut into tiles of tile_x * tile_y nodes; the
// flattened tile list is walked round-robin by all CTAs of a grid sized to the
// number of co-resident CTAs (cooperative launch), so uneven instance sizes
// balance out.  Between time steps the CTAs meet at a device-wide barrier whose
// waits are bounded in time: a wait that runs out records an error and every
// CTA leaves the kernel, which the host reports as DDFLB_ETIMEOUT.
//
// Every check_every steps the step kernel also accumulates, per tile, the sums
// for the velocity residual r = |u(t) - u(t-1)|_2 / |u(t)|_2 and the mass;
// after a barrier each instance's tiles are reduced in a fixed order
// (deterministic), and an instance whose residual fell below the tolerance or
// whose sums are not finite is frozen (its tiles are skipped from then on).
//
// The chunk launch reads the current step from device memory, so one captured
// CUDA graph of the launch replays for every chunk.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/ddflb.h"
#include "ddflb_device.cuh"
#include "ddflb_internal.h"

namespace ddflb {

// per-tile sums of a check: |u|^2, |u - u_prev|^2, rho - rho0, phi^2, (phi - phi_prev)^2
constexpr int kParts = 5;
// tile descriptors a CTA keeps in shared memory when its range is this short
constexpr int kTileCache = 64;

struct BatchInst {
  LbParams P;
  void* buf[2];  // f planes; g planes follow 9 planes later
  float* uprev;  // 3 planes [ny][nx]: u_x, u_y, phi
  int64_t goff;  // element offset of the g planes from the f planes
  int32_t tile_begin, tile_end;
  int32_t bc;
  int32_t pad;
};

struct BatchStatus {
  double residual;      // the residual the freeze decision uses
  double residual_phi;  // |phi(t) - phi(t-K)| / (K |phi(t)|)
  double u2;
  double mass_dev;
  int64_t steps_to_tol;  // state time at which the residual first fell below tol (-1: not yet)
  int64_t state_time;    // state time of the instance's current state when frozen
  long long init_time;   // state time at which the instance was (re)initialised
  int32_t flags;         // DDFLB_INST_CONVERGED | DDFLB_INST_DIVERGED | DDFLB_INST_CAPPED
  int32_t pad;
  double tol;            // this instance's tolerance (< 0: the batch's)
  int64_t max_steps;     // freeze after this many steps since init (0: no limit)
};

struct BatchSync {
  unsigned word;  // barrier counter (see grid_barrier)
  unsigned pad0;
  int err;        // 1: a barrier wait ran out (sticky until the batch is reset)
  int pad;
  int64_t step;  // state time of all active instances
  int64_t pad2[5];
};

struct BatchArgs {
  const BatchInst* inst;
  int ninst;
  const int4* tiles;
  int ntiles;
  int tile_x, tile_y;
  int nsteps;
  int check_every;
  double tol;
  int scalar_residual;  // freeze only when the scalar residual is below tol too
  double* part;  // kParts doubles per tile
  BatchStatus* ist;
  BatchSync* sync;
  long long timeout_ns;
  int skip_block;  // test hook: this CTA never arrives at the first barrier (-1: none)
};

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Device-wide barrier for a cooperative grid (all CTAs co-resident), on one
// sense-reversing 32-bit counter: CTA 0 adds 2^31 - (N - 1), every other CTA
// adds 1, so each barrier adds exactly 2^31.  The top bit therefore flips at
// the last of the N arrivals, whatever their order, and cannot flip back
// before all N have arrived at the next barrier.  Each CTA makes one acq_rel
// atomic (releasing its writes) and polls with acquire loads until the top bit
// differs from the value its atomic returned.  Returns false if the barrier
// failed: this CTA's wait ran out, or another CTA's did (the sticky error word,
// read every 32 polls, then stops everyone).
__device__ bool grid_barrier(BatchSync* s, long long timeout_ns) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;"
                 : "=r"(old)
                 : "l"(&s->word), "r"(add)
                 : "memory");
    const unsigned long long t0 = now_ns();
    unsigned spins = 0;
    int good = 1;
    while (((ld_acquire(&s->word) ^ old) & 0x80000000u) == 0u) {
      if ((++spins & 31u) == 0u) {
        if (*(volatile int*)&s->err != 0) {
          good = 0;
          break;
        }
        // the spin count bounds the wait independently of the timer
        if ((long long)(now_ns() - t0) > timeout_ns || spins > (1u << 28)) {
          atomicExch(&s->err, 1);
          good = 0;
          break;
        }
      }
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// Residual sums of one node at a check step (against the snapshot taken K
// steps earlier), then its new snapshot (velocity and scalar).
__device__ __forceinline__ void node_sums(const LbParams& P, const BatchInst& I, int x, int y,
                                          const Mom& mf, const Macro& q, bool snap, bool check,
                                          double acc[kParts]) {
  const int64_t c = (int64_t)y * P.nx + x, n = (int64_t)P.nx * P.ny;
  if (check) {
    const double ex = (double)q.ux - I.uprev[c], ey = (double)q.uy - I.uprev[n + c];
    const double ep = (double)q.phi - I.uprev[2 * n + c];
    acc[0] += (double)q.ux * q.ux + (double)q.uy * q.uy;
    acc[1] += ex * ex + ey * ey;
    acc[2] += (double)mf.k0;
    acc[3] += (double)q.phi * q.phi;
    acc[4] += ep * ep;
  }
  if (snap) {
    I.uprev[c] = q.ux;
    I.uprev[n + c] = q.uy;
    I.uprev[2 * n + c] = q.phi;
  }
}

// COH: load through L2 only (the persistent kernel, whose planes other CTAs
// rewrite within the launch); otherwise the read-only path (one step a launch)
// SUMS: also the residual sums and the snapshot (at check steps); the
// per-step schedule leaves them to k_batch_sums.
template <typename S, int BC, bool COH, bool SUMS = true>
__device__ __forceinline__ void batch_cell(const LbParams& P, const BatchInst& I, int src, int x,
                                           int y, bool inner, bool snap, bool check,
                                           double acc[kParts]) {
  const S* fin = (const S*)I.buf[src];
  const S* gin = fin + I.goff;
  S* fout = (S*)I.buf[src ^ 1];
  S* gout = fout + I.goff;
  float df[9], dg[9];
  // a warp whose nodes all have their 8 neighbours inside the lattice pulls
  // without the wall rules (same addresses, so the same values)
  if (BC != BC_PERIODIC && inner)
    pull<S, BC_PERIODIC, COH>(P, fin, gin, x, y, df, dg);
  else
    pull<S, BC, COH>(P, fin, gin, x, y, df, dg);
  const Mom mf = moments_flow(df), mg = moments_scalar(dg);
  const Macro q = macro(P, mf, mg);
  Neq nf = neq_flow(mf, q), ng = neq_scalar(P, mg, mf, q);
  // FP32 storage: compensated odd moments, as in the single-lattice step
  if (sizeof(S) == 4) neq_compensate<false>(P, df, dg, mf, mg, q, 0.0f, 0.0f, nf, ng);
  relax(P.wf, nf, df);
  relax(P.wg, ng, dg);
  const uint32_t o = (uint32_t)y * (uint32_t)P.pitch + (uint32_t)x;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    Codec<S>::store(fout + a * P.plane + o, df[a], P.sf);
    Codec<S>::store(gout + a * P.plane + o, dg[a], P.sg);
  }
  if (SUMS && (check || snap)) node_sums(P, I, x, y, mf, q, snap, check, acc);
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < nw; ++k) t += sh[k];
  return t;  // valid in thread 0
}

// Check of instance i after the step from state time t (a multiple of K): the
// fixed-order reduction of its tiles' sums, then the freeze decision
// (converged, diverged, or at its own step limit).  Called by one whole CTA.
__device__ void check_instance(const BatchArgs& A, int i, int64_t t, double* sh) {
  if (__ldcg(&A.ist[i].flags) != 0 || t - A.check_every < __ldcg(&A.ist[i].init_time)) return;
  const int b = A.inst[i].tile_begin, e = A.inst[i].tile_end;
  double v[kParts];
  for (int k = 0; k < kParts; ++k) {
    double a = 0.0;
    for (int j = b + threadIdx.x; j < e; j += blockDim.x) a += __ldcg(&A.part[kParts * (int64_t)j + k]);
    v[k] = block_sum(a, sh);
  }
  if (threadIdx.x == 0) {
    BatchStatus& st = A.ist[i];
    st.u2 = v[0];
    st.mass_dev = v[2];
    const double ru = v[0] > 0.0 ? sqrt(v[1] / v[0]) / A.check_every : 0.0;
    const double rp = v[3] > 0.0 ? sqrt(v[4] / v[3]) / A.check_every : 0.0;
    st.residual_phi = rp;
    st.residual = A.scalar_residual ? fmax(ru, rp) : ru;
    const double tol = st.tol >= 0.0 ? st.tol : A.tol;
    if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2]) || !isfinite(v[3])) {
      st.flags = DDFLB_INST_DIVERGED;
      st.state_time = t + 1;
    } else if (tol > 0.0 && st.residual < tol) {
      st.flags = DDFLB_INST_CONVERGED;
      st.steps_to_tol = t - st.init_time;  // steps since this instance's init
      st.state_time = t + 1;
    } else if (st.max_steps > 0 && t + 1 - st.init_time >= st.max_steps) {
      st.flags = DDFLB_INST_CAPPED;  // its own step limit, without convergence
      st.state_time = t + 1;
    }
  }
}

// At most 64 registers a thread (4 CTAs of 256 threads or 8 of 128 per SM):
// the step is latency-bound on memory, so resident warps matter more than the
// few values that spill.  BCS: the boundary kind of every instance, when they
// all share one (the kernel then carries only that pull), else -1 (chosen per
// tile at run time).
template <typename S, int BCS>
__global__ void __launch_bounds__(256, 4) k_batch(BatchArgs A) {
  __shared__ BatchInst sI;
  __shared__ double sh[8];
  __shared__ int sActive;
  __shared__ long long sInit;
  const int64_t t0 = A.sync->step;
  const LbParams& sP = sI.P;
  // each CTA owns a contiguous range of tiles: instance parameters are staged
  // in shared memory once per instance change, not once per tile
  const int per = (A.ntiles + gridDim.x - 1) / gridDim.x;
  const int tb = blockIdx.x * per, te = min(A.ntiles, tb + per);
  // a short tile range is read once into shared memory, so a step of small
  // lattices does not wait on an L2 load of the tile descriptor per tile
  __shared__ int4 sTiles[kTileCache];
  const bool cached = te - tb <= kTileCache;
  if (cached)
    for (int k = threadIdx.x; k < te - tb; k += blockDim.x) sTiles[k] = A.tiles[tb + k];
  __syncthreads();
  const int tx = threadIdx.x % A.tile_x, ty = threadIdx.x / A.tile_x;  // place in the tile
  int cur = -1;
  for (int s = 0; s < A.nsteps; ++s) {
    const int64_t t = t0 + s;
    const int src = (int)(t & 1);
    // at every multiple of K: compare u with the snapshot from K steps earlier
    // (instances initialised at least K steps ago), then take the next snapshot
    const bool snap = A.check_every > 0 && t % A.check_every == 0;
    const bool check_t = snap && t > 0;
    for (int tile = tb; tile < te; ++tile) {
      const int4 T = cached ? sTiles[tile - tb] : A.tiles[tile];
      if (T.x != cur) {
        __syncthreads();
        const int* srcw = (const int*)(A.inst + T.x);
        int* dstw = (int*)&sI;
        for (int w = threadIdx.x; w < (int)(sizeof(BatchInst) / 4); w += blockDim.x) dstw[w] = srcw[w];
        if (threadIdx.x == 0) {
          sActive = __ldcg(&A.ist[T.x].flags) == 0;
          sInit = __ldcg(&A.ist[T.x].init_time);
        }
        cur = T.x;
        __syncthreads();
      }
      if (!sActive) continue;
      const bool check = check_t && t - A.check_every >= sInit;
      const int x = T.y + tx, y = T.z + ty;
      double acc[kParts] = {0.0, 0.0, 0.0, 0.0, 0.0};
      // warp-uniform (all lanes vote, before any lane drops out); the channel is
      // periodic in x, so only its walls in y count
      const bool in_x = sI.bc == BC_CHANNEL ? x < sP.nx : (x >= 1 && x < sP.nx - 1);
      const bool inner = __all_sync(0xffffffffu, in_x && y >= 1 && y < sP.ny - 1);
      if (x < sP.nx && y < sP.ny) {
        if (BCS >= 0) {
          batch_cell<S, (BCS >= 0 ? BCS : 0), true>(sP, sI, src, x, y, inner, snap, check, acc);
        } else {
          switch (sI.bc) {
            case BC_PERIODIC:
              batch_cell<S, BC_PERIODIC, true>(sP, sI, src, x, y, inner, snap, check, acc);
              break;
            case BC_CAVITY:
              batch_cell<S, BC_CAVITY, true>(sP, sI, src, x, y, inner, snap, check, acc);
              break;
            default: batch_cell<S, BC_CHANNEL, true>(sP, sI, src, x, y, inner, snap, check, acc);
          }
        }
      }
      if (check) {
        for (int k = 0; k < kParts; ++k) {
          const double v = block_sum(acc[k], sh);
          if (threadIdx.x == 0) A.part[kParts * (int64_t)tile + k] = v;
        }
      }
    }
    if (check_t) {
      if (!grid_barrier(A.sync, A.timeout_ns)) return;
      for (int i = blockIdx.x; i < A.ninst; i += gridDim.x) check_instance(A, i, t, sh);
      cur = -1;  // re-read the activity flags
    }
    if (s == 0 && (int)blockIdx.x == A.skip_block) return;  // test hook: never arrive
    if (!grid_barrier(A.sync, A.timeout_ns)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) A.sync->step = t0 + A.nsteps;
}

// Schedule 1: one ordinary launch per time step, one CTA per tile, then (idle
// except at check steps) the sums and check kernels and, at the end of a
// chunk, the state-time update, all captured in one graph per chunk.  No
// device-wide barrier: the stream orders the steps.  Step s of the chunk
// advances the state from time sync->step + s.  The node update carries no
// check code; at most 56 registers, so 9 CTAs of 128 threads stay resident.
template <typename S>
__global__ void __maxnreg__(56) k_batch_tile(BatchArgs A, int s) {
  __shared__ BatchInst sI;
  __shared__ int sActive;
  const int64_t t = A.sync->step + s;
  const int4 T = __ldg(&A.tiles[blockIdx.x]);
  const int* srcw = (const int*)(A.inst + T.x);
  int* dstw = (int*)&sI;
  for (int w = threadIdx.x; w < (int)(sizeof(BatchInst) / 4); w += blockDim.x) dstw[w] = __ldg(&srcw[w]);
  if (threadIdx.x == 0) sActive = __ldcg(&A.ist[T.x].flags) == 0;
  __syncthreads();
  if (!sActive) return;  // uniform over the CTA
  const LbParams& sP = sI.P;
  const int src = (int)(t & 1);
  const int tx = threadIdx.x % A.tile_x, ty = threadIdx.x / A.tile_x;
  const int x = T.y + tx, y = T.z + ty;
  const bool in_x = sI.bc == BC_CHANNEL ? x < sP.nx : (x >= 1 && x < sP.nx - 1);
  const bool inner = __all_sync(0xffffffffu, in_x && y >= 1 && y < sP.ny - 1);
  if (x >= sP.nx || y >= sP.ny) return;
  double none[kParts];
  switch (sI.bc) {
    case BC_PERIODIC:
      batch_cell<S, BC_PERIODIC, false, false>(sP, sI, src, x, y, inner, false, false, none);
      break;
    case BC_CAVITY:
      batch_cell<S, BC_CAVITY, false, false>(sP, sI, src, x, y, inner, false, false, none);
      break;
    default: batch_cell<S, BC_CHANNEL, false, false>(sP, sI, src, x, y, inner, false, false, none);
  }
}

// At a check step (state time t a multiple of K, after the step from t): the
// residual sums of each tile from the state at time t, read back from the
// step's source buffer (the step wrote the other one), and the new snapshot.
// A grid of a few CTAs per SM walks the tiles; at other steps it returns.
template <typename S>
__global__ void __launch_bounds__(256) k_batch_sums(BatchArgs A, int s) {
  __shared__ BatchInst sI;
  __shared__ double sh[8];
  __shared__ int sActive;
  __shared__ long long sInit;
  const int64_t t = A.sync->step + s;
  const bool snap = A.check_every > 0 && t % A.check_every == 0;
  if (!snap) return;
  const LbParams& sP = sI.P;
  const int src = (int)(t & 1);
  const int tx = threadIdx.x % A.tile_x, ty = threadIdx.x / A.tile_x;
  int cur = -1;
  for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
    const int4 T = __ldg(&A.tiles[tile]);
    if (T.x != cur) {
      __syncthreads();
      const int* srcw = (const int*)(A.inst + T.x);
      int* dstw = (int*)&sI;
      for (int w = threadIdx.x; w < (int)(sizeof(BatchInst) / 4); w += blockDim.x) dstw[w] = __ldg(&srcw[w]);
      if (threadIdx.x == 0) {
        // the flag as it was before this step's check (the check kernel runs next)
        sActive = __ldcg(&A.ist[T.x].flags) == 0;
        sInit = __ldcg(&A.ist[T.x].init_time);
      }
      cur = T.x;
      __syncthreads();
    }
    if (!sActive) continue;
    const bool check = t > 0 && t - A.check_every >= sInit;
    const int x = T.y + tx, y = T.z + ty;
    double acc[kParts] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (x < sP.nx && y < sP.ny) {
      const S* fin = (const S*)sI.buf[src];
      float df[9], dg[9];
      switch (sI.bc) {
        case BC_PERIODIC: pull<S, BC_PERIODIC>(sP, fin, fin + sI.goff, x, y, df, dg); break;
        case BC_CAVITY: pull<S, BC_CAVITY>(sP, fin, fin + sI.goff, x, y, df, dg); break;
        default: pull<S, BC_CHANNEL>(sP, fin, fin + sI.goff, x, y, df, dg);
      }
      const Mom mf = moments_flow(df), mg = moments_scalar(dg);
      node_sums(sP, sI, x, y, mf, macro(sP, mf, mg), true, check, acc);
    }
    if (check) {
      for (int k = 0; k < kParts; ++k) {
        const double v = block_sum(acc[k], sh);
        if (threadIdx.x == 0) A.part[kParts * (int64_t)tile + k] = v;
      }
    }
  }
}

// The checks after step s of a chunk (a no-op unless its state time is a
// positive multiple of K): one CTA per instance.
__global__ void __launch_bounds__(256) k_batch_check(BatchArgs A, int s) {
  __shared__ double sh[8];
  const int64_t t = A.sync->step + s;
  if (!(A.check_every > 0 && t > 0 && t % A.check_every == 0)) return;
  check_instance(A, blockIdx.x, t, sh);
}

__global__ void k_batch_advance(BatchSync* sync, int nsteps) {
  if (threadIdx.x == 0) sync->step += nsteps;
}

}  // namespace ddflb

using namespace ddflb;

namespace {

thread_local std::string g_berr;

ddflb_status bfail(ddflb_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_error(buf);
  return s;
}

ddflb_status bcuda(cudaError_t e, const char* where) {
  return bfail(DDFLB_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

constexpr size_t kAl = 256;
size_t al(size_t v) { return (v + kAl - 1) / kAl * kAl; }
size_t esz(int storage) { return storage == DDFLB_FP32 ? 4 : 2; }
int bpitch(int nx) { return (nx + 31) / 32 * 32; }

const int kShapes[][2] = {{32, 4}, {64, 2}, {128, 1}, {32, 8}, {64, 4}, {128, 2}, {256, 1}};
constexpr int kNumShapes = 7;

struct BLayout {
  std::vector<size_t> off_buf0, off_buf1, off_uprev;
  size_t off_inst, off_tiles, off_part, off_status, off_sync, total;
  int max_tiles;
};

int count_tiles(int n, const ddflb_params* p, int tx, int ty) {
  int64_t t = 0;
  for (int i = 0; i < n; ++i) t += (int64_t)((p[i].nx + tx - 1) / tx) * ((p[i].ny + ty - 1) / ty);
  return t > (1 << 30) ? -1 : (int)t;
}

BLayout blayout(int n, const ddflb_params* p) {
  BLayout L;
  size_t o = 0;
  for (int i = 0; i < n; ++i) {
    const size_t plane = (size_t)bpitch(p[i].nx) * p[i].ny;
    const size_t bytes = al(18 * plane * esz(p[i].storage));
    L.off_buf0.push_back(o); o += bytes;
    L.off_buf1.push_back(o); o += bytes;
    L.off_uprev.push_back(o); o += al(3 * (size_t)p[i].nx * p[i].ny * sizeof(float));
  }
  int mt = 0;
  for (int k = 0; k < kNumShapes; ++k) mt = std::max(mt, count_tiles(n, p, kShapes[k][0], kShapes[k][1]));
  L.max_tiles = mt;
  L.off_inst = o; o += al(n * sizeof(BatchInst));
  L.off_tiles = o; o += al((size_t)mt * sizeof(int4));
  L.off_part = o; o += al((size_t)mt * kParts * sizeof(double));
  L.off_status = o; o += al(n * sizeof(BatchStatus));
  L.off_sync = o; o += al(sizeof(BatchSync));
  L.total = o;
  return L;
}

}  // namespace

struct ddflb_batch {
  int n;
  std::vector<ddflb_params> p;
  std::vector<LbParams> lp;
  BLayout lay;
  char* ws;
  cudaStream_t stream;
  int storage;
  int tile_x, tile_y, blocks_per_sm, grid;
  int ntiles;
  int chunk;
  double tol;
  int scalar_residual;
  long long timeout_ns;
  int skip_block;
  int64_t step;  // host mirror of the global state time
  BatchInst* d_inst;
  int4* d_tiles;
  double* d_part;
  BatchStatus* d_status;
  BatchSync* d_sync;
  cudaGraphExec_t graph;
  int graph_chunk;
  bool graph_failed;
  std::vector<double> inst_tol;   // per-instance tolerance (< 0: the batch's)
  std::vector<int64_t> inst_cap;  // per-instance step limit (0: none)
  int schedule;                   // 0 persistent cooperative launch, 1 one launch per step
  int bcs;                        // the boundary kind all instances share, or -1
  int sums_grid;                  // CTAs of the check-step sums kernel (schedule 1)
};

namespace {

ddflb_status upload_tiles(ddflb_batch* b) {
  std::vector<int4> tiles;
  std::vector<BatchInst> inst(b->n);
  for (int i = 0; i < b->n; ++i) {
    BatchInst& I = inst[i];
    std::memset(&I, 0, sizeof I);
    I.P = b->lp[i];
    I.buf[0] = b->ws + b->lay.off_buf0[i];
    I.buf[1] = b->ws + b->lay.off_buf1[i];
    I.uprev = (float*)(b->ws + b->lay.off_uprev[i]);
    I.goff = 9 * I.P.plane;
    I.bc = b->p[i].bc;
    I.tile_begin = (int)tiles.size();
    for (int y = 0; y < b->p[i].ny; y += b->tile_y)
      for (int x = 0; x < b->p[i].nx; x += b->tile_x) tiles.push_back(make_int4(i, x, y, 0));
    I.tile_end = (int)tiles.size();
  }
  b->ntiles = (int)tiles.size();
  cudaError_t e = cudaMemcpyAsync(b->d_inst, inst.data(), inst.size() * sizeof(BatchInst),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? DDFLB_OK : bcuda(e, "batch tile upload");
}

template <typename S>
void* kernel_ptr(int schedule, int bcs) {
  if (schedule == 1) return (void*)k_batch_tile<S>;
  return bcs == BC_PERIODIC ? (void*)k_batch<S, BC_PERIODIC>
       : bcs == BC_CAVITY   ? (void*)k_batch<S, BC_CAVITY>
       : bcs == BC_CHANNEL  ? (void*)k_batch<S, BC_CHANNEL>
                            : (void*)k_batch<S, -1>;
}

// bcs: the boundary kind all instances share, or -1
void* batch_kernel(int storage, int schedule, int bcs) {
  return storage == 0 ? kernel_ptr<float>(schedule, bcs)
                      : storage == 1 ? kernel_ptr<__half>(schedule, bcs)
                                     : kernel_ptr<__nv_bfloat16>(schedule, bcs);
}

ddflb_status configure(ddflb_batch* b, int tx, int ty, int bps) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int occ = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel(b->storage, b->schedule, b->bcs),
                                                      tx * ty, 0);
  if (e != cudaSuccess) return bcuda(e, "batch occupancy");
  if (occ < 1) return bfail(DDFLB_EINVAL, "batch kernel cannot be resident with %d threads", tx * ty);
  b->tile_x = tx;
  b->tile_y = ty;
  b->blocks_per_sm = bps > 0 ? std::min(bps, occ) : occ;
  b->grid = b->blocks_per_sm * nsm;
  b->sums_grid = 4 * nsm;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return upload_tiles(b);
}

BatchArgs args_for(ddflb_batch* b, int nsteps) {
  BatchArgs A;
  A.inst = b->d_inst;
  A.ninst = b->n;
  A.tiles = b->d_tiles;
  A.ntiles = b->ntiles;
  A.tile_x = b->tile_x;
  A.tile_y = b->tile_y;
  A.nsteps = nsteps;
  A.check_every = b->p[0].check_every;
  A.tol = b->tol;
  A.scalar_residual = b->scalar_residual;
  A.part = b->d_part;
  A.ist = b->d_status;
  A.sync = b->d_sync;
  A.timeout_ns = b->timeout_ns;
  A.skip_block = b->skip_block;
  return A;
}

cudaError_t launch_chunk(ddflb_batch* b, cudaStream_t s, int nsteps) {
  BatchArgs A = args_for(b, nsteps);
  if (b->schedule == 1) {
    // one launch per step (+ the check kernel), then the state-time update
    const dim3 tb(b->tile_x * b->tile_y);
    void* sums = b->storage == 0 ? (void*)k_batch_sums<float>
               : b->storage == 1 ? (void*)k_batch_sums<__half> : (void*)k_batch_sums<__nv_bfloat16>;
    for (int k = 0; k < nsteps; ++k) {
      void* targs[] = {&A, &k};
      cudaError_t e = cudaLaunchKernel(batch_kernel(b->storage, 1, b->bcs), dim3(b->ntiles), tb, targs, 0, s);
      if (e == cudaSuccess) e = cudaLaunchKernel(sums, dim3(b->sums_grid), tb, targs, 0, s);
      if (e != cudaSuccess) return e;
      k_batch_check<<<b->n, 256, 0, s>>>(A, k);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    k_batch_advance<<<1, 32, 0, s>>>(b->d_sync, nsteps);
    return cudaGetLastError();
  }
  void* kargs[] = {&A};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(b->tile_x * b->tile_y);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, batch_kernel(b->storage, 0, b->bcs), kargs);
}

// Capture one chunk launch into a graph (on a private stream) for replay.
void build_graph(ddflb_batch* b, int nsteps) {
  if (b->graph_failed) return;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    b->graph_failed = true;
    return;
  }
  cudaGraph_t g = nullptr;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    ok = launch_chunk(b, cs, nsteps) == cudaSuccess;
    ok = (cudaStreamEndCapture(cs, &g) == cudaSuccess) && ok;
  }
  cudaGraphExec_t ex = nullptr;
  if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  cudaGetLastError();  // clear a capture error, if any
  if (!ok) {
    b->graph_failed = true;
    return;
  }
  b->graph = ex;
  b->graph_chunk = nsteps;
}

ddflb_status check_sync_error(ddflb_batch* b) {
  BatchSync h;
  cudaError_t e = cudaMemcpyAsync(&h, b->d_sync, sizeof h, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch status");
  if (h.err) return bfail(DDFLB_ETIMEOUT, "a device-wide barrier wait ran out (step %lld)",
                          (long long)h.step);
  return DDFLB_OK;
}

}  // namespace

extern "C" {

size_t ddflb_batch_workspace_bytes(int32_t n, const ddflb_params* p) {
  if (n <= 0 || !p) return 0;
  for (int i = 0; i < n; ++i) {
    if (ddflb_workspace_bytes(&p[i]) == 0) return 0;
    if (p[i].scalar_model >= DDFLB_SCALAR_CASCADED) {
      set_error("the batched step runs the MRT and SRT scalar collisions only");
      return 0;
    }
    if (p[i].fx != 0.0 || p[i].fy != 0.0 || p[i].force_omega != 0.0) {
      set_error("the batched step runs unforced instances only (fx = fy = force_omega = 0)");
      return 0;
    }
    if (p[i].storage != p[0].storage || p[i].check_every != p[0].check_every) {
      set_error("all instances of a batch share storage and check_every");
      return 0;
    }
  }
  const BLayout L = blayout(n, p);
  return L.max_tiles < 0 ? 0 : L.total;
}

ddflb_status ddflb_batch_create(int32_t n, const ddflb_params* p, void* ws, size_t bytes,
                                void* stream, ddflb_batch** out) {
  if (!out) return bfail(DDFLB_EINVAL, "out is NULL");
  *out = nullptr;
  const size_t need = ddflb_batch_workspace_bytes(n, p);
  if (need == 0) return DDFLB_EINVAL;  // message set by the size query
  if (!ws || (uintptr_t)ws % kAl) return bfail(DDFLB_EINVAL, "workspace NULL or not 256-aligned");
  if (bytes < need) return bfail(DDFLB_ENOMEM, "workspace %zu bytes < %zu required", bytes, need);
  ddflb_batch* b = new (std::nothrow) ddflb_batch();
  if (!b) return bfail(DDFLB_ENOMEM, "host allocation of the handle failed");
  b->n = n;
  b->p.assign(p, p + n);
  b->lay = blayout(n, p);
  for (int i = 0; i < n; ++i) b->lp.push_back(make_lbparams(&p[i], bpitch(p[i].nx)));
  b->ws = (char*)ws;
  b->stream = (cudaStream_t)stream;
  b->storage = p[0].storage;
  b->bcs = p[0].bc;
  for (int i = 1; i < n; ++i)
    if (p[i].bc != p[0].bc) b->bcs = -1;
  b->chunk = 500;
  b->tol = 0.0;
  b->timeout_ns = 2000000000LL;
  b->skip_block = -1;
  b->step = 0;
  b->d_inst = (BatchInst*)(b->ws + b->lay.off_inst);
  b->d_tiles = (int4*)(b->ws + b->lay.off_tiles);
  b->d_part = (double*)(b->ws + b->lay.off_part);
  b->d_status = (BatchStatus*)(b->ws + b->lay.off_status);
  b->d_sync = (BatchSync*)(b->ws + b->lay.off_sync);
  b->graph = nullptr;
  b->graph_failed = false;
  b->schedule = 0;
  cudaError_t e = cudaMemsetAsync(b->d_sync, 0, sizeof(BatchSync), b->stream);
  if (e != cudaSuccess) {
    delete b;
    return bcuda(e, "batch create");
  }
  b->inst_tol.assign(n, -1.0);
  b->inst_cap.assign(n, 0);
  std::vector<BatchStatus> st(n);
  for (auto& s : st) {
    std::memset(&s, 0, sizeof s);
    s.steps_to_tol = -1;
    s.residual = NAN;
    s.tol = -1.0;
  }
  e = cudaMemcpyAsync(b->d_status, st.data(), n * sizeof(BatchStatus), cudaMemcpyHostToDevice,
                      b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    delete b;
    return bcuda(e, "batch create");
  }
  ddflb_status s = configure(b, 128, 1, 0);
  if (s != DDFLB_OK) {
    delete b;
    return s;
  }
  *out = b;
  return DDFLB_OK;
}

ddflb_status ddflb_batch_set_run(ddflb_batch* b, double tol, int32_t steps_per_launch,
                                 double barrier_timeout_s, int32_t scalar_residual) {
  if (!b) return bfail(DDFLB_EINVAL, "NULL batch");
  if (!(tol >= 0) || steps_per_launch < 1 || !(barrier_timeout_s > 0 && barrier_timeout_s <= 60))
    return bfail(DDFLB_EINVAL, "tol >= 0, steps_per_launch >= 1, timeout in (0, 60] s");
  b->tol = tol;
  b->scalar_residual = scalar_residual != 0;
  b->chunk = steps_per_launch;
  b->timeout_ns = (long long)(barrier_timeout_s * 1e9);
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return DDFLB_OK;
}

ddflb_status ddflb_batch_set_instance_run(ddflb_batch* b, int32_t i, double tol,
                                          int64_t max_steps) {
  if (!b || i < 0 || i >= b->n) return bfail(DDFLB_EINVAL, "bad batch or instance index");
  if (!(tol == tol) || max_steps < 0) return bfail(DDFLB_EINVAL, "tol is NaN or max_steps < 0");
  b->inst_tol[i] = tol;
  b->inst_cap[i] = max_steps;
  // also into the live status (takes effect at the next check; the rest of
  // the status is left as it is)
  BatchStatus* d = b->d_status + i;
  cudaError_t e = cudaMemcpyAsync(&d->tol, &b->inst_tol[i], sizeof(double),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&d->max_steps, &b->inst_cap[i], sizeof(int64_t), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? DDFLB_OK : bcuda(e, "batch instance run");
}

ddflb_status ddflb_batch_set_schedule(ddflb_batch* b, int32_t schedule) {
  if (!b) return bfail(DDFLB_EINVAL, "NULL batch");
  if (schedule != 0 && schedule != 1) return bfail(DDFLB_EINVAL, "schedule must be 0 or 1");
  b->schedule = schedule;
  return configure(b, b->tile_x, b->tile_y, schedule == 1 ? 0 : b->blocks_per_sm);
}

ddflb_status ddflb_batch_get_schedule(const ddflb_batch* b, int32_t* schedule) {
  if (!b || !schedule) return bfail(DDFLB_EINVAL, "NULL argument");
  *schedule = b->schedule;
  return DDFLB_OK;
}

ddflb_status ddflb_batch_set_tiles(ddflb_batch* b, int32_t tile_x, int32_t tile_y,
                                   int32_t blocks_per_sm) {
  if (!b) return bfail(DDFLB_EINVAL, "NULL batch");
  bool ok = false;
  for (int k = 0; k < kNumShapes; ++k) ok = ok || (kShapes[k][0] == tile_x && kShapes[k][1] == tile_y);
  if (!ok) return bfail(DDFLB_EINVAL, "tile %d x %d is not one of the supported shapes", tile_x, tile_y);
  if (blocks_per_sm < 0) return bfail(DDFLB_EINVAL, "blocks_per_sm < 0");
  return configure(b, tile_x, tile_y, blocks_per_sm);
}

ddflb_status ddflb_batch_get_tiles(const ddflb_batch* b, int32_t* tile_x, int32_t* tile_y,
                                   int32_t* blocks_per_sm) {
  if (!b) return bfail(DDFLB_EINVAL, "NULL batch");
  if (tile_x) *tile_x = b->tile_x;
  if (tile_y) *tile_y = b->tile_y;
  if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
  return DDFLB_OK;
}

ddflb_status ddflb_batch_init(ddflb_batch* b, int32_t i, const float* rho, const float* ux,
                              const float* uy, const float* phi, const float* grads) {
  if (!b || i < 0 || i >= b->n || !rho || !ux || !uy || !phi)
    return bfail(DDFLB_EINVAL, "bad batch, instance index or NULL field");
  const ddflb_params& p = b->p[i];
  if (grads && (p.omega_f[3] <= 0 || p.omega_f[4] <= 0 || p.omega_f[5] <= 0 ||
                p.omega_g[1] <= 0 || p.omega_g[2] <= 0 || p.omega_g[5] <= 0))
    return bfail(DDFLB_EINVAL, "gradient initialisation needs w3, w4, w5, w1^phi, w2^phi, w5^phi > 0");
  Launch L;
  L.P = b->lp[i];
  L.P_bc = p.bc;
  L.storage = p.storage;
  L.force = false;
  L.block = dim3(128, 1, 1);
  L.stream = b->stream;
  InitPtrs in{rho, ux, uy, phi, grads};
  // the instance joins at the batch's current state time
  const size_t off = (b->step & 1) ? b->lay.off_buf1[i] : b->lay.off_buf0[i];
  char* f = b->ws + off;
  char* g = f + 9 * (size_t)L.P.plane * esz(p.storage);
  cudaError_t e = launch_init(L, in, f, g);
  if (e != cudaSuccess) return bcuda(e, "batch init");
  BatchStatus s;
  std::memset(&s, 0, sizeof s);
  s.steps_to_tol = -1;
  s.residual = NAN;
  s.init_time = b->step;
  s.tol = b->inst_tol[i];
  s.max_steps = b->inst_cap[i];
  e = cudaMemcpyAsync(b->d_status + i, &s, sizeof s, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? DDFLB_OK : bcuda(e, "batch init status");
}

ddflb_status ddflb_batch_step(ddflb_batch* b, int64_t n) {
  if (!b) return bfail(DDFLB_EINVAL, "NULL batch");
  if (n < 0) return bfail(DDFLB_EINVAL, "n < 0");
  // one NVTX range over the call's chunk launches (graph replays)
  nvtxRangePushA("ddflb_batch_step");
  struct PopRange {
    ~PopRange() { nvtxRangePop(); }
  } pop_range;
  int64_t left = n;
  while (left > 0) {
    const int k = (int)std::min<int64_t>(left, b->chunk);
    if (k == b->chunk && !b->graph) build_graph(b, k);
    cudaError_t e;
    if (k == b->chunk && b->graph)
      e = cudaGraphLaunch(b->graph, b->stream);
    else
      e = launch_chunk(b, b->stream, k);
    if (e != cudaSuccess) return bcuda(e, "batch step launch");
    left -= k;
    b->step += k;
  }
  return DDFLB_OK;
}

ddflb_status ddflb_batch_fields(ddflb_batch* b, int32_t i, float* rho, float* ux, float* uy,
                                float* phi, float* sxx, float* sxy, float* syy, float* omega) {
  if (!b || i < 0 || i >= b->n) return bfail(DDFLB_EINVAL, "bad batch or instance index");
  BatchStatus s;
  cudaError_t e = cudaMemcpyAsync(&s, b->d_status + i, sizeof s, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch fields status");
  const int64_t t = s.flags ? s.state_time : b->step;
  Launch L;
  L.P = b->lp[i];
  L.P_bc = b->p[i].bc;
  L.storage = b->p[i].storage;
  L.force = false;
  L.block = dim3(128, 1, 1);
  L.stream = b->stream;
  const char* f = b->ws + ((t & 1) ? b->lay.off_buf1[i] : b->lay.off_buf0[i]);
  const char* g = f + 9 * (size_t)L.P.plane * esz(b->p[i].storage);
  FieldPtrs fp{{rho, ux, uy, phi, sxx, sxy, syy, omega}};
  e = launch_fields(L, f, g, fp);
  return e == cudaSuccess ? DDFLB_OK : bcuda(e, "batch fields");
}

ddflb_status ddflb_batch_stats(ddflb_batch* b, double* residual, int32_t* flags,
                               int64_t* steps_to_tol, int64_t* state_time, int64_t* init_time) {
  if (!b) return bfail(DDFLB_EINVAL, "NULL batch");
  std::vector<BatchStatus> h(b->n);
  cudaError_t e = cudaMemcpyAsync(h.data(), b->d_status, b->n * sizeof(BatchStatus),
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch stats");
  for (int i = 0; i < b->n; ++i) {
    if (residual) residual[i] = h[i].residual;
    if (flags) flags[i] = h[i].flags;
    if (steps_to_tol) steps_to_tol[i] = h[i].steps_to_tol;
    if (state_time) state_time[i] = h[i].flags ? h[i].state_time : b->step;
    if (init_time) init_time[i] = h[i].init_time;
  }
  return check_sync_error(b);
}

ddflb_status ddflb_batch_debug_skip_barrier(ddflb_batch* b, int32_t block) {
  if (!b) return bfail(DDFLB_EINVAL, "NULL batch");
  b->skip_block = block;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return DDFLB_OK;
}

// Autotuner: times every supported tile shape at full and half residency on
// the batch itself (CUDA events on the batch stream, one untimed launch then
// one timed launch of trial_steps each) and keeps the fastest.  The trials run
// on zeroed populations (the rest state), so this overwrites every instance's
// state: call it before ddflb_batch_init.
ddflb_status ddflb_batch_autotune(ddflb_batch* b, int32_t trial_steps, int32_t* tile_x,
                                  int32_t* tile_y, int32_t* blocks_per_sm, double* ms_per_step) {
  if (!b || trial_steps < 1) return bfail(DDFLB_EINVAL, "NULL batch or trial_steps < 1");
  cudaStream_t s = b->stream;
  cudaError_t e = cudaMemsetAsync(b->ws, 0, b->lay.off_inst, s);
  if (e != cudaSuccess) return bcuda(e, "autotune clear");
  std::vector<BatchStatus> st(b->n);
  for (auto& x : st) {
    std::memset(&x, 0, sizeof x);
    x.steps_to_tol = -1;
    x.residual = NAN;
    x.tol = -1.0;  // during the trials: the batch tolerance, 0 (nothing freezes)
  }
  e = cudaMemcpyAsync(b->d_status, st.data(), b->n * sizeof(BatchStatus), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return bcuda(e, "autotune status");
  const double tol = b->tol;
  b->tol = 0.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bx = 128, by = 1, bb = 0, bs = 0;
  ddflb_status rs = DDFLB_OK;
  const int saved_schedule = b->schedule;
  // candidates per tile shape: the persistent launch at full and half
  // residency (variant 0, 1), and one launch per step (variant 2)
  for (int k = 0; k < kNumShapes && rs == DDFLB_OK; ++k) {
    for (int half = 0; half < 3 && rs == DDFLB_OK; ++half) {
      b->schedule = half == 2 ? 1 : 0;
      rs = configure(b, kShapes[k][0], kShapes[k][1], 0);
      if (rs != DDFLB_OK) break;
      if (half == 1) {
        if (b->blocks_per_sm < 2) continue;
        rs = configure(b, kShapes[k][0], kShapes[k][1], b->blocks_per_sm / 2);
        if (rs != DDFLB_OK) break;
      }
      e = launch_chunk(b, s, trial_steps);
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = launch_chunk(b, s, trial_steps);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        rs = bcuda(e, "autotune trial");
        break;
      }
      if (ms < best) {
        best = ms;
        bx = b->tile_x;
        by = b->tile_y;
        bb = b->blocks_per_sm;
        bs = b->schedule;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tol = tol;
  if (rs != DDFLB_OK) {
    b->schedule = saved_schedule;
    return rs;
  }
  b->schedule = bs;
  rs = configure(b, bx, by, bb);
  if (rs != DDFLB_OK) return rs;
  // back to a clean state at time 0, with the per-instance run settings
  for (int i = 0; i < b->n; ++i) {
    st[i].tol = b->inst_tol[i];
    st[i].max_steps = b->inst_cap[i];
  }
  e = cudaMemsetAsync(b->ws, 0, b->lay.off_inst, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_sync, 0, sizeof(BatchSync), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_status, st.data(), b->n * sizeof(BatchStatus), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bcuda(e, "autotune reset");
  b->step = 0;
  if (tile_x) *tile_x = bx;
  if (tile_y) *tile_y = by;
  if (blocks_per_sm) *blocks_per_sm = bb;
  if (ms_per_step) *ms_per_step = best / trial_steps;
  return DDFLB_OK;
}

ddflb_status ddflb_batch_destroy(ddflb_batch* b) {
  if (b && b->graph) cudaGraphExecDestroy(b->graph);
  delete b;
  return DDFLB_OK;
}

}  // extern "C"
