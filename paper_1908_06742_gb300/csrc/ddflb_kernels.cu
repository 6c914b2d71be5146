// Kernels of the fused DDF lattice Boltzmann step for sm_103a, and their
// launchers (host side, internal to the library).
//
//   k_step      one time step: pull both lattices with the wall rules, moments,
//               MRT collision of both, back-transform, store (Secs. 2, 3, 5)
//   k_fields    local kinematics of the current state (Sec. 4), optionally the
//               full velocity gradient, scalar gradient, Q, R and Lamb vector
//   k_pops      current pre-collision populations as full values
//   k_init      equilibrium + Chapman-Enskog non-equilibrium initial state,
//               written in the pre-streamed layout the pull step expects
//   k_reduce    FP64 sums (mass, scalar, |u|^2, |u - u_prev|^2) per block
//   k_finalize  fixed-order sum of the block partials into the status block
//
// The step is a memory-bound stencil: 18 populations read and 18 written per
// node (144 B at FP32 storage), about 300 FP32 operations; no tensor cores.
#include <cuda_runtime.h>

#include "ddflb_device.cuh"
#include "ddflb_internal.h"

namespace ddflb {

// ------------------------------------------------------------------ step
// At most 56 registers a thread: 9 blocks of 128 threads stay resident per SM
// (59 registers would allow 8).  The step waits on memory, so the extra warps
// pay: measured 1.002 against 0.978 of the copy peak at 16384^2 FP32, with
// no spills (48 registers spill and run at 0.93).
template <typename S, int BC, bool FORCE, int SM>
__global__ void __maxnreg__(56) k_step(LbParams P, const S* __restrict__ fin,
                                              const S* __restrict__ gin, S* __restrict__ fout,
                                              S* __restrict__ gout,
                                              const DevStatus* __restrict__ status) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = P.y0 + blockIdx.y * blockDim.y + threadIdx.y;
  // with walls: a warp (32 consecutive x of one row) whose nodes all have their
  // neighbours inside the buffers pulls without the wall rules (same addresses,
  // same values); decided by a vote of all lanes before any returns
  bool inner = false;
  if (BC != BC_PERIODIC) {
    const bool in_x = BC == BC_CHANNEL ? x < P.nx : (x >= 1 && x < P.nx - 1);
    inner = __all_sync(0xffffffffu, in_x && y >= 1 && y < P.ny - 1);
  }
  if (x >= P.nx || y >= P.y1) return;
  if (status != nullptr && status->diverged) return;
  float df[9], dg[9];
  if (BC != BC_PERIODIC && inner)
    pull<S, BC_PERIODIC>(P, fin, gin, x, y, df, dg);
  else
    pull<S, BC>(P, fin, gin, x, y, df, dg);
  // FP32 storage: compensated odd moments (the arithmetic rounding would
  // otherwise match the storage rounding); 16-bit storage rounds far coarser
  collide<FORCE, SM, sizeof(S) == 4>(P, x, y, df, dg);
  const uint32_t o = (uint32_t)y * (uint32_t)P.pitch + (uint32_t)x;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    Codec<S>::store(fout + a * P.plane + o, df[a], P.sf);
    Codec<S>::store(gout + a * P.plane + o, dg[a], P.sg);
  }
}

// ------------------------------------------------------------------ fields
template <typename S, int BC, bool FORCE>
__global__ void __launch_bounds__(256) k_fields(LbParams P, const S* __restrict__ fin,
                                                const S* __restrict__ gin, FieldPtrs out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = P.y0 + blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= P.nx || y >= P.y1) return;
  float df[9], dg[9];
  pull<S, BC>(P, fin, gin, x, y, df, dg);
  Neq nf, ng;
  const Macro q = state<FORCE>(P, x, y, df, dg, nf, ng);
  const Kin k = kinematics(P, nf, ng, q);
  const int64_t o = (int64_t)(y - P.y0) * P.nx + x;
  if (out.p[0]) out.p[0][o] = q.rho;
  if (out.p[1]) out.p[1][o] = q.ux;
  if (out.p[2]) out.p[2][o] = q.uy;
  if (out.p[3]) out.p[3][o] = q.phi;
  if (out.p[4]) out.p[4][o] = k.sxx;
  if (out.p[5]) out.p[5][o] = k.sxy;
  if (out.p[6]) out.p[6][o] = k.syy;
  if (out.p[7]) out.p[7][o] = k.omega;
  if (out.derived) {
    const Inv v = invariants(k, q);
    const float d[10] = {k.sxx, k.dyux, k.dxuy, k.syy, k.dxphi, k.dyphi, v.q, v.r, v.lx, v.ly};
#pragma unroll
    for (int i = 0; i < 10; ++i)
      if (out.p[8 + i]) out.p[8 + i][o] = d[i];
  }
}

// ------------------------------------------------------------------ populations
template <typename S, int BC>
__global__ void __launch_bounds__(256) k_pops(LbParams P, const S* __restrict__ fin,
                                              const S* __restrict__ gin, float* __restrict__ fo,
                                              float* __restrict__ go) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = P.y0 + blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= P.nx || y >= P.y1) return;
  float df[9], dg[9];
  pull<S, BC>(P, fin, gin, x, y, df, dg);
  const int64_t o = (int64_t)(y - P.y0) * P.nx + x, n = (int64_t)P.nx * (P.y1 - P.y0);
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    if (fo) fo[a * n + o] = df[a] + P.wrf[a] * P.rho0;
    if (go) go[a * n + o] = dg[a] + P.wrg[a] * P.phi0;
  }
}

// ------------------------------------------------------------------ init
// Node (x, y) builds its populations at t = 0 and scatters them to the slots
// the first pull will read: direction a goes to the upstream node x - e_a if
// that node exists (periodic wrap included), otherwise (a wall link) into the
// node's own slot of the opposite direction, with the wall rule undone.
template <typename S, int BC, bool FORCE>
__global__ void __launch_bounds__(256) k_init(LbParams P, InitPtrs in, S* __restrict__ fout,
                                              S* __restrict__ gout) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = P.y0 + blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= P.nx || y >= P.y1) return;
  const int64_t c0 = (int64_t)(y - P.y0) * P.nx + x, n = (int64_t)P.nx * (P.y1 - P.y0);
  const float rho = in.rho[c0], ux = in.ux[c0], uy = in.uy[c0], phi = in.phi[c0];
  const float k0 = rho - P.rho0, n0 = phi - P.phi0;
  const float jx = rho * ux, jy = rho * uy, px = phi * ux, py = phi * uy;
  const float c = 1.0f / 3.0f, uxx = ux * ux, uyy = uy * uy, usq = uxx + uyy;
  // equilibrium moments, Eqs. (eqmrawmoment), (eqmrawmoment_CDE), deviation form
  float m3 = 2.0f * c * k0 + rho * usq, m4 = rho * (uxx - uyy), m5 = jx * uy;
  float e1 = px, e2 = py, e3 = 2.0f * c * n0 + phi * usq, e4 = phi * (uxx - uyy), e5 = px * uy;
  float e6 = py * (P.b1 * c + uxx), e7 = px * (P.b2 * c + uyy);
  float e8 = c * c * n0 + phi * (c * usq + uxx * uyy);
  const bool cm = P.smodel >= 2;  // central-moment scalar models (Apps. C, D)
  // their equilibrium is the raw image of the central equilibria: larger in
  // the fourth-order moment by 2 c phi ((b2 - 1) ux^2 + (b1 - 1) uy^2)
  if (cm) e8 += 2.0f * c * phi * ((P.b2 - 1.0f) * uxx + (P.b1 - 1.0f) * uyy);
  if (in.grads) {
    // Chapman-Enskog non-equilibrium parts: Eqs. (strainratexxpyy)-(strainratexy)
    // for the flow; Eqs. (1stnoneqmmomentx_CDE), (1stnoneqmmomenty_CDE),
    // (offdiagonal2ndnoneqmmoment_CDE) for the scalar.
    const float dxux = in.grads[c0], dyux = in.grads[n + c0];
    const float dxuy = in.grads[2 * n + c0], dyuy = in.grads[3 * n + c0];
    const float dxph = in.grads[4 * n + c0], dyph = in.grads[5 * n + c0];
    m3 += -2.0f * c * rho / P.wf[3] * (dxux + dyuy);
    m4 += -2.0f * c * rho / P.wf[4] * (dxux - dyuy);
    m5 += -c * rho / P.wf[5] * (dxuy + dyux);
    const float Nphi = phi * (P.b1 * dxuy + P.b2 * dyux);
    const float vx = -c / P.wg[1] * dxph, vy = -c / P.wg[2] * dyph;
    if (!cm) {
      e1 += vx;
      e2 += vy;
      e5 += -c / P.wg[5] * (Nphi + P.b1 * uy * dxph + P.b2 * ux * dyph);
    } else {
      // central non-equilibrium parts (x, y and xy), taken to raw moments by the
      // inverse binomial shift: eta_xy^(1) = -(c / w5)[phi N^phi + (b1 - 1) uy
      // dxphi + (b2 - 1) ux dyphi]
      const float vxy =
          -c / P.wg[5] * (Nphi + (P.b1 - 1.0f) * uy * dxph + (P.b2 - 1.0f) * ux * dyph);
      e1 += vx;
      e2 += vy;
      e3 += 2.0f * (ux * vx + uy * vy);
      e4 += 2.0f * (ux * vx - uy * vy);
      e5 += vxy + uy * vx + ux * vy;
      e6 += 2.0f * ux * vxy + uxx * vy + 2.0f * ux * uy * vx;
      e7 += 2.0f * uy * vxy + uyy * vx + 2.0f * ux * uy * vy;
      e8 += 2.0f * uxx * uy * vy + 2.0f * ux * uyy * vx + 4.0f * ux * uy * vxy;
    }
  }
  float m1 = jx, m2 = jy, m6 = jy * (c + uxx), m7 = jx * (c + uyy);
  float m8 = c * c * k0 + rho * (c * usq + uxx * uyy);
  if (FORCE) {
    // the flow populations held are f-bar = f - S/2, S at the force of t = 0
    const Macro v{rho, 0.0f, ux, uy, phi};
    const Src s = source(node_force(P, x, y), v);
    m1 -= 0.5f * s.s1;
    m2 -= 0.5f * s.s2;
    m3 -= 0.5f * s.s3;
    m4 -= 0.5f * s.s4;
    m5 -= 0.5f * s.s5;
    m6 -= 0.5f * s.s6;
    m7 -= 0.5f * s.s7;
    m8 -= 0.5f * s.s8;
  }
  float df[9], dg[9];
  populations(k0, m1, m2, m3, m4, m5, m6, m7, m8, df);
  populations(n0, e1, e2, e3, e4, e5, e6, e7, e8, dg);
  constexpr int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  constexpr int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    int zx = x - ex[a], zy = y - ey[a];
    bool wall = false, lid = false;
    if (BC == BC_CAVITY) wall = zx < 0 || zx >= P.nx;
    if (BC == BC_PERIODIC) {
      zy = (zy + P.ny) % P.ny;
    } else {
      lid = zy >= P.ny;
      wall = wall || zy < 0 || lid;
    }
    if (BC != BC_CAVITY) zx = (zx + P.nx) % P.nx;
    if (!wall) {
      const int64_t o = a * P.plane + (int64_t)zy * P.pitch + zx;
      Codec<S>::store(fout + o, df[a], P.sf);
      Codec<S>::store(gout + o, dg[a], P.sg);
    } else {
      const int64_t o = opp[a] * P.plane + (int64_t)y * P.pitch + x;
      const float vf = df[a] - (lid ? P.lid[a] : 0.0f);
      const float vg = (lid ? P.abb_lid[a] : P.abb_wall[a]) - dg[a];
      Codec<S>::store(fout + o, vf, P.sf);
      Codec<S>::store(gout + o, vg, P.sg);
    }
  }
}

// ------------------------------------------------------------------ reductions
// mode bit 1: compute |u - u_prev|^2 against the snapshot; bit 2: write the
// current u as the new snapshot.  Partials: 4 doubles per block.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <typename S, int BC, bool FORCE>
__global__ void __launch_bounds__(kReduceThreads) k_reduce(LbParams P, const S* __restrict__ fin,
                                                           const S* __restrict__ gin,
                                                           float* __restrict__ uprev, int mode,
                                                           double* __restrict__ partials) {
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t n = (int64_t)P.nx * (P.y1 - P.y0);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(c / P.nx), x = (int)(c - (int64_t)r * P.nx), y = P.y0 + r;
    float df[9], dg[9];
    pull<S, BC>(P, fin, gin, x, y, df, dg);
    Mom mf = moments_flow(df);
    const Mom mg = moments_scalar(dg);
    const Macro q = FORCE ? macro_force(P, mf, mg, node_force(P, x, y)) : macro(P, mf, mg);
    s[0] += (double)mf.k0;
    s[1] += (double)mg.k0;
    s[2] += (double)q.ux * q.ux + (double)q.uy * q.uy;
    if (mode & 1) {
      const double ex = (double)q.ux - uprev[c], ey = (double)q.uy - uprev[n + c];
      s[3] += ex * ex + ey * ey;
    }
    if (mode & 2) {
      uprev[c] = q.ux;
      uprev[n + c] = q.uy;
    }
  }
  __shared__ double sh[kReduceThreads / 32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double v = warp_sum(s[k]);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < kReduceThreads / 32; ++w) t += sh[w][threadIdx.x];
    partials[4 * blockIdx.x + threadIdx.x] = t;
  }
}

// One block: thread k sums partials k, k + 256, ... (fixed order), then a
// fixed tree.  mode bit 1: this reduction is a residual check.
__global__ void __launch_bounds__(256) k_finalize(const double* __restrict__ partials, int nparts,
                                                  int mode, DevStatus* __restrict__ st) {
  __shared__ double sh[4][256];
  for (int k = 0; k < 4; ++k) {
    double t = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 256) t += partials[4 * i + k];
    sh[k][threadIdx.x] = t;
  }
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->mass_dev = sh[0][0];
    st->scalar_dev = sh[1][0];
    st->u2 = sh[2][0];
    if (mode & 1) {
      st->du2 = sh[3][0];
      st->residual = sh[2][0] > 0.0 ? sqrt(sh[3][0] / sh[2][0]) : 0.0;
      st->has_residual = 1;
    }
    if (!isfinite(sh[0][0]) || !isfinite(sh[1][0]) || !isfinite(sh[2][0])) st->diverged = 1;
  }
}

// ------------------------------------------------------------------ y-slab halos
// A lattice divided into y-slabs (the collide-and-stream update of Secs. 2-3
// is local: a node pulls only from its 8 neighbours) exchanges, after every
// step, the post-collision populations that cross each shared face: the
// directions with e_y = -1 (4, 7, 8) of a slab's bottom row go down, those
// with e_y = +1 (2, 5, 6) of its top row go up, for both lattices: 6 rows of
// nx storage elements per face and direction, copied bit for bit (E is an
// unsigned integer of the storage element's size).
__device__ __forceinline__ int halo_plane(int k, bool up) {
  const int a = k % 3;
  return up ? (a == 0 ? 2 : a == 1 ? 5 : 6) : (a == 0 ? 4 : a == 1 ? 7 : 8);
}

// message rows [6][nx]: k = 0..2 flow, 3..5 scalar
template <typename E>
__global__ void __launch_bounds__(256) k_halo_pack(LbParams P, const E* __restrict__ buf,
                                                   int64_t gofs, E* __restrict__ down,
                                                   E* __restrict__ up) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
  if (x >= P.nx) return;
  const E* lat = buf + (k >= 3 ? gofs : 0);
  if (down) down[k * P.nx + x] = lat[halo_plane(k, false) * P.plane + (int64_t)P.y0 * P.pitch + x];
  if (up) up[k * P.nx + x] = lat[halo_plane(k, true) * P.plane + (int64_t)(P.y1 - 1) * P.pitch + x];
}

template <typename E>
__global__ void __launch_bounds__(256) k_halo_unpack(LbParams P, E* __restrict__ buf, int64_t gofs,
                                                     const E* __restrict__ from_below,
                                                     const E* __restrict__ from_above) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
  if (x >= P.nx) return;
  E* lat = buf + (k >= 3 ? gofs : 0);
  if (from_below)  // ghost row below the slab receives what the slab below sent up
    lat[halo_plane(k, true) * P.plane + (int64_t)(P.y0 - 1) * P.pitch + x] = from_below[k * P.nx + x];
  if (from_above)
    lat[halo_plane(k, false) * P.plane + (int64_t)P.y1 * P.pitch + x] = from_above[k * P.nx + x];
}

// All faces of slabs on one device in one launch: block z = 2 s + dir copies
// slab s's outgoing rows straight into the ghost row of its neighbour (dir 0:
// up to slab s + 1, dir 1: down to slab s - 1; wrapping for a periodic lattice).
template <typename E>
__global__ void __launch_bounds__(256) k_halo_local(HaloSlabs H) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
  const int s = blockIdx.z >> 1;
  const bool up = (blockIdx.z & 1) == 0;
  const int t = up ? s + 1 : s - 1;
  if (x >= H.nx) return;
  const int d = t < 0 ? (H.periodic ? H.n - 1 : -1) : t >= H.n ? (H.periodic ? 0 : -1) : t;
  if (d < 0) return;
  const HaloSlab& A = H.s[s];
  const HaloSlab& B = H.s[d];
  const int a = halo_plane(k, up);
  const int64_t lat = k >= 3 ? 1 : 0;
  const E* src = (const E*)A.buf + lat * A.gofs_elems + a * A.plane;
  E* dst = (E*)B.buf + lat * B.gofs_elems + a * B.plane;
  const int64_t ys = up ? A.y1 - 1 : A.y0, yd = up ? B.y0 - 1 : B.y1;
  dst[yd * H.pitch + x] = src[ys * H.pitch + x];
}

// ------------------------------------------------------------------ launchers
namespace {
dim3 grid2d(const LbParams& P, dim3 b) {
  return dim3((P.nx + b.x - 1) / b.x, (P.y1 - P.y0 + b.y - 1) / b.y);
}

template <typename S, int BC, bool FORCE, int SM>
cudaError_t run(const Launch& L, int what, const void* fin, const void* gin, void* a, void* b,
                const FieldPtrs* fp, const InitPtrs* ip, int mode, double* partials, int nparts,
                const DevStatus* st) {
  const dim3 blk = L.block, g = grid2d(L.P, blk);
  switch (what) {
    case 0:
      k_fields<S, BC, FORCE><<<g, blk, 0, L.stream>>>(L.P, (const S*)fin, (const S*)gin, *fp);
      break;
    case 1:
      k_pops<S, BC><<<g, blk, 0, L.stream>>>(L.P, (const S*)fin, (const S*)gin, (float*)a,
                                             (float*)b);
      break;
    case 2:
      k_init<S, BC, FORCE><<<g, blk, 0, L.stream>>>(L.P, *ip, (S*)a, (S*)b);
      break;
    case 3:
      k_reduce<S, BC, FORCE><<<nparts, kReduceThreads, 0, L.stream>>>(
          L.P, (const S*)fin, (const S*)gin, (float*)a, mode, partials);
      break;
    default:
      k_step<S, BC, FORCE, SM><<<g, blk, 0, L.stream>>>(L.P, (const S*)fin, (const S*)gin,
                                                        (S*)a, (S*)b, st);
  }
  return cudaGetLastError();
}

// scalar model: the step kernel is specialised (0 MRT / SRT, 2 cascaded, 3 central
// moments); the other kernels read P.smodel where it matters
template <typename S, int BC, bool FORCE>
cudaError_t run_sm(const Launch& L, int what, const void* fin, const void* gin, void* a, void* b,
                   const FieldPtrs* fp, const InitPtrs* ip, int mode, double* partials, int np,
                   const DevStatus* st) {
  if (what != 4 || L.P.smodel < 2)
    return run<S, BC, FORCE, 0>(L, what, fin, gin, a, b, fp, ip, mode, partials, np, st);
  if (L.P.smodel == 2)
    return run<S, BC, FORCE, 2>(L, what, fin, gin, a, b, fp, ip, mode, partials, np, st);
  return run<S, BC, FORCE, 3>(L, what, fin, gin, a, b, fp, ip, mode, partials, np, st);
}

template <typename S, int BC>
cudaError_t run_f(const Launch& L, int what, const void* fin, const void* gin, void* a, void* b,
                  const FieldPtrs* fp, const InitPtrs* ip, int mode, double* partials, int np,
                  const DevStatus* st) {
  if (L.force) return run_sm<S, BC, true>(L, what, fin, gin, a, b, fp, ip, mode, partials, np, st);
  return run_sm<S, BC, false>(L, what, fin, gin, a, b, fp, ip, mode, partials, np, st);
}

template <typename S>
cudaError_t run_bc(const Launch& L, int what, const void* fin, const void* gin, void* a, void* b,
                   const FieldPtrs* fp, const InitPtrs* ip, int mode, double* partials, int np,
                   const DevStatus* st) {
  switch (L.P_bc) {
    case BC_PERIODIC:
      return run_f<S, BC_PERIODIC>(L, what, fin, gin, a, b, fp, ip, mode, partials, np, st);
    case BC_CAVITY:
      return run_f<S, BC_CAVITY>(L, what, fin, gin, a, b, fp, ip, mode, partials, np, st);
    default:
      return run_f<S, BC_CHANNEL>(L, what, fin, gin, a, b, fp, ip, mode, partials, np, st);
  }
}

cudaError_t dispatch(const Launch& L, int what, const void* fin, const void* gin, void* a, void* b,
                     const FieldPtrs* fp, const InitPtrs* ip, int mode, double* partials, int np,
                     const DevStatus* st = nullptr) {
  switch (L.storage) {
    case 0: return run_bc<float>(L, what, fin, gin, a, b, fp, ip, mode, partials, np, st);
    case 1: return run_bc<__half>(L, what, fin, gin, a, b, fp, ip, mode, partials, np, st);
    default: return run_bc<__nv_bfloat16>(L, what, fin, gin, a, b, fp, ip, mode, partials, np, st);
  }
}
}  // namespace

cudaError_t launch_step(const Launch& L, const void* fin, const void* gin, void* fout, void* gout,
                        const DevStatus* st) {
  return dispatch(L, 4, fin, gin, fout, gout, nullptr, nullptr, 0, nullptr, 0, st);
}

cudaError_t launch_fields(const Launch& L, const void* fin, const void* gin, const FieldPtrs& out) {
  return dispatch(L, 0, fin, gin, nullptr, nullptr, &out, nullptr, 0, nullptr, 0);
}

cudaError_t launch_pops(const Launch& L, const void* fin, const void* gin, float* f, float* g) {
  return dispatch(L, 1, fin, gin, f, g, nullptr, nullptr, 0, nullptr, 0);
}

cudaError_t launch_init(const Launch& L, const InitPtrs& in, void* fout, void* gout) {
  return dispatch(L, 2, nullptr, nullptr, fout, gout, nullptr, &in, 0, nullptr, 0);
}

cudaError_t launch_halo_pack(const Launch& L, const void* buf, size_t gofs_bytes, void* down,
                             void* up) {
  const dim3 b(256), g((L.P.nx + 255) / 256, 6);
  if (L.storage == 0)
    k_halo_pack<uint32_t><<<g, b, 0, L.stream>>>(L.P, (const uint32_t*)buf, gofs_bytes / 4,
                                                 (uint32_t*)down, (uint32_t*)up);
  else
    k_halo_pack<uint16_t><<<g, b, 0, L.stream>>>(L.P, (const uint16_t*)buf, gofs_bytes / 2,
                                                 (uint16_t*)down, (uint16_t*)up);
  return cudaGetLastError();
}

cudaError_t launch_halo_unpack(const Launch& L, void* buf, size_t gofs_bytes,
                               const void* from_below, const void* from_above) {
  const dim3 b(256), g((L.P.nx + 255) / 256, 6);
  if (L.storage == 0)
    k_halo_unpack<uint32_t><<<g, b, 0, L.stream>>>(L.P, (uint32_t*)buf, gofs_bytes / 4,
                                                   (const uint32_t*)from_below,
                                                   (const uint32_t*)from_above);
  else
    k_halo_unpack<uint16_t><<<g, b, 0, L.stream>>>(L.P, (uint16_t*)buf, gofs_bytes / 2,
                                                   (const uint16_t*)from_below,
                                                   (const uint16_t*)from_above);
  return cudaGetLastError();
}

cudaError_t launch_halo_local(const HaloSlabs& H, int storage, cudaStream_t stream) {
  const dim3 b(256), g((H.nx + 255) / 256, 6, 2 * H.n);
  if (storage == 0)
    k_halo_local<uint32_t><<<g, b, 0, stream>>>(H);
  else
    k_halo_local<uint16_t><<<g, b, 0, stream>>>(H);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const Launch& L, const void* fin, const void* gin, float* uprev,
                          int mode, double* partials, DevStatus* st) {
  cudaError_t e = dispatch(L, 3, fin, gin, uprev, nullptr, nullptr, nullptr, mode, partials,
                           kReduceBlocks);
  if (e != cudaSuccess) return e;
  k_finalize<<<1, 256, 0, L.stream>>>(partials, kReduceBlocks, mode, st);
  return cudaGetLastError();
}

}  // namespace ddflb
