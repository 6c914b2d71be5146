// Fused step for 16-bit population storage with several adjacent nodes per
// thread (this file: two, k_step_pair, and four, k_step_quad).
//
// With FP16/BF16 storage a one-node-per-thread pull moves 2 bytes per memory
// access; 36 such streams per node reach only about 0.7 of the HBM copy
// bandwidth even with no arithmetic (4-byte accesses about 0.83, aligned
// 8-byte accesses about 0.93).  In k_step_pair each thread owns the pair of
// nodes (x0, x0 + 1), x0 even: every plane is read as aligned 4-byte pairs; a
// plane pulled from x - 1 or x + 1 also reads the aligned pair to the left
// (x0 - 2) or right (x0 + 2), whose other half the neighbouring thread reads as
// well (served from L1); stores are 4-byte pairs.  The per-node arithmetic is
// exactly that of k_step (same device functions), so results are
// bit-identical to the one-node kernel.
//
// Requirements: nx even (k_step_pair), nx a multiple of 4 (k_step_quad).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "ddflb_device.cuh"
#include "ddflb_internal.h"

namespace ddflb {

template <typename S> struct PairOf;
template <> struct PairOf<__half> {
  typedef __half2 T;
  static __device__ __forceinline__ float lo(T v) { return __low2float(v); }
  static __device__ __forceinline__ float hi(T v) { return __high2float(v); }
  static __device__ __forceinline__ T pack(float a, float b) { return __floats2half2_rn(a, b); }
  static __device__ __forceinline__ T zero() { return __floats2half2_rn(0.f, 0.f); }
};
template <> struct PairOf<__nv_bfloat16> {
  typedef __nv_bfloat162 T;
  static __device__ __forceinline__ float lo(T v) { return __low2float(v); }
  static __device__ __forceinline__ float hi(T v) { return __high2float(v); }
  static __device__ __forceinline__ T pack(float a, float b) { return __floats2bfloat162_rn(a, b); }
  static __device__ __forceinline__ T zero() { return __floats2bfloat162_rn(0.f, 0.f); }
};

template <typename S>
__device__ __forceinline__ typename PairOf<S>::T ld_pair(const S* p) {
  typedef typename PairOf<S>::T T;
  unsigned v = __ldg(reinterpret_cast<const unsigned*>(p));
  return *reinterpret_cast<T*>(&v);
}

template <typename S>
__device__ __forceinline__ void st_pair(S* p, float a, float b, float s) {
  typedef typename PairOf<S>::T T;
  T v = PairOf<S>::pack(a * s, b * s);
  __stcs(reinterpret_cast<unsigned*>(p), *reinterpret_cast<unsigned*>(&v));
}

template <typename S, int BC>
__global__ void __launch_bounds__(256) k_step_pair(LbParams P, const S* __restrict__ fin,
                                                   const S* __restrict__ gin, S* __restrict__ fout,
                                                   S* __restrict__ gout,
                                                   const DevStatus* __restrict__ status) {
  typedef PairOf<S> Q;
  constexpr int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  constexpr int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (y >= P.ny) return;  // whole warps share y
  if (status != nullptr && status->diverged) return;
  const int nx = P.nx, ny = P.ny;
  const int64_t pl = P.plane;
  const bool live = x0 < nx;
  int ym = y - 1, yp = y + 1;
  bool sym = false, syp = false;
  if (BC == BC_PERIODIC) {
    if (ym < 0) ym += ny;
    if (yp >= ny) yp -= ny;
  } else {
    sym = ym < 0;
    syp = yp >= ny;
  }
  // the aligned pairs left and right of the own pair (x0 - 2 holds node A's
  // source x0 - 1, x0 + 2 node B's source x0 + 2); beyond a wall: none
  int xl2 = x0 - 2, xr2 = x0 + 2;
  bool sxl = false, sxr = false;
  if (BC == BC_CAVITY) {
    sxl = xl2 < 0;
    sxr = xr2 >= nx;
  } else {
    if (xl2 < 0) xl2 += nx;
    if (xr2 >= nx) xr2 -= nx;
  }
  const int64_t rows[3] = {(int64_t)ym * P.pitch, (int64_t)y * P.pitch, (int64_t)yp * P.pitch};
  const int64_t own = (int64_t)y * P.pitch + x0;
  float fA[9], fB[9], gA[9], gB[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const int ex = EX[a], ey = EY[a];
    const bool ysolid = (ey == 1 && sym) || (ey == -1 && syp);
    const int64_t ro = rows[1 - ey];
    typename Q::T fp = Q::zero(), gp = Q::zero();
    if (live && !ysolid) {
      fp = ld_pair(fin + a * pl + ro + x0);
      gp = ld_pair(gin + a * pl + ro + x0);
    }
    float fa, fb, ga, gb;
    if (ex == 0) {
      fa = Q::lo(fp); fb = Q::hi(fp); ga = Q::lo(gp); gb = Q::hi(gp);
    } else if (ex == 1) {  // source x - 1: node A from the high half of pair x0 - 2
      typename Q::T fl = Q::zero(), gl = Q::zero();
      if (live && !ysolid && !sxl) {
        fl = ld_pair(fin + a * pl + ro + xl2);
        gl = ld_pair(gin + a * pl + ro + xl2);
      }
      fa = Q::hi(fl); fb = Q::lo(fp); ga = Q::hi(gl); gb = Q::lo(gp);
    } else {  // source x + 1: node B from the low half of pair x0 + 2
      typename Q::T fr = Q::zero(), gr = Q::zero();
      if (live && !ysolid && !sxr) {
        fr = ld_pair(fin + a * pl + ro + xr2);
        gr = ld_pair(gin + a * pl + ro + xr2);
      }
      fa = Q::hi(fp); fb = Q::lo(fr); ga = Q::hi(gp); gb = Q::lo(gr);
    }
    fA[a] = fa * P.isf; fB[a] = fb * P.isf; gA[a] = ga * P.isg; gB[a] = gb * P.isg;
    if (BC != BC_PERIODIC) {
      // half-way bounce-back: the node's own post-collision value of the
      // opposite direction, with the moving-wall / fixed-scalar terms
      const bool solA = ysolid || (ex == 1 && sxl);
      const bool solB = ysolid || (ex == -1 && sxr);
      if ((solA || solB) && live) {
        const typename Q::T fo = ld_pair(fin + OPP[a] * pl + own);
        const typename Q::T go = ld_pair(gin + OPP[a] * pl + own);
        const bool lid = ey == -1 && syp;
        const float lf = lid ? P.lid[a] : 0.0f;
        const float lg = lid ? P.abb_lid[a] : P.abb_wall[a];
        if (solA) {
          fA[a] = Q::lo(fo) * P.isf + lf;
          gA[a] = lg - Q::lo(go) * P.isg;
        }
        if (solB) {
          fB[a] = Q::hi(fo) * P.isf + lf;
          gB[a] = lg - Q::hi(go) * P.isg;
        }
      }
    }
  }
  if (!live) return;
  {
    const Mom mf = moments_flow(fA), mg = moments_scalar(gA);
    const Macro q = macro(P, mf, mg);
    relax(P.wf, neq_flow(mf, q), fA);
    relax(P.wg, neq_scalar(P, mg, mf, q), gA);
  }
  {
    const Mom mf = moments_flow(fB), mg = moments_scalar(gB);
    const Macro q = macro(P, mf, mg);
    relax(P.wf, neq_flow(mf, q), fB);
    relax(P.wg, neq_scalar(P, mg, mf, q), gB);
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    st_pair(fout + a * pl + own, fA[a], fB[a], P.sf);
    st_pair(gout + a * pl + own, gA[a], gB[a], P.sg);
  }
}

// Four adjacent nodes per thread (x0 .. x0 + 3, x0 a multiple of 4) on a
// lattice with nx a multiple of 4: every plane is read as one aligned 8-byte
// group; a plane pulled from x - 1 (x + 1) also reads the group to the left
// (right), of which node x0 (x0 + 3) takes the last (first) element.  The four
// nodes are collided one after another with k_step's device functions and
// stored as 8-byte groups.  A group with a node next to a wall (rows 0 and
// ny - 1; for the cavity also the first and last group of a row) steps its
// nodes one by one with k_step's pull and wall rules instead.  Bit-identical to
// the one-node kernel.
template <typename S>
__device__ __forceinline__ uint2 ld_quad(const S* p) {
  return __ldg(reinterpret_cast<const uint2*>(p));
}
template <typename S> __device__ __forceinline__ float half_of(unsigned w, int hi);
template <> __device__ __forceinline__ float half_of<__half>(unsigned w, int hi) {
  return __half2float(__ushort_as_half((unsigned short)(hi ? w >> 16 : w & 0xffffu)));
}
// a BF16 value is the upper half of its FP32 value: one mask or shift
template <> __device__ __forceinline__ float half_of<__nv_bfloat16>(unsigned w, int hi) {
  return __uint_as_float(hi ? w & 0xffff0000u : w << 16);
}
// element k (0..3) of an 8-byte group
template <typename S> __device__ __forceinline__ float elem(uint2 v, int k) {
  return half_of<S>(k < 2 ? v.x : v.y, k & 1);
}
// two values already in storage units as one packed word (lo in the low half),
// one paired round-to-nearest conversion: the same bits as converting each alone
template <typename S> __device__ __forceinline__ unsigned pack2(float lo, float hi);
template <> __device__ __forceinline__ unsigned pack2<__half>(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&h);
}
template <> __device__ __forceinline__ unsigned pack2<__nv_bfloat16>(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&h);
}

// At most 96 registers a thread: 5 CTAs of 128 threads per SM instead of 4 at
// the unconstrained 126, for a few bytes of spills (measured at 16384^2: FP16
// 0.92 against 0.87 of the copy peak, BF16 0.89 against 0.85).
template <typename S, int BC>
__global__ void __maxnreg__(96) k_step_quad(LbParams P, const S* __restrict__ fin,
                                                   const S* __restrict__ gin,
                                                   S* __restrict__ fout, S* __restrict__ gout,
                                                   const DevStatus* __restrict__ status) {
  constexpr int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x0 >= P.nx || y >= P.ny) return;
  if (status != nullptr && status->diverged) return;
  const int nx = P.nx, ny = P.ny;
  const int64_t pl = P.plane;
  if (BC != BC_PERIODIC &&
      (y == 0 || y == ny - 1 || (BC == BC_CAVITY && (x0 == 0 || x0 + 4 == nx)))) {
    // next to a wall: node by node, as k_step
    const uint32_t o0 = (uint32_t)y * (uint32_t)P.pitch + (uint32_t)x0;
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
      float df[9], dg[9];
      pull<S, BC>(P, fin, gin, x0 + k, y, df, dg);
      collide<false, 0>(P, x0 + k, y, df, dg);
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        Codec<S>::store(fout + a * pl + (o0 + k), df[a], P.sf);
        Codec<S>::store(gout + a * pl + (o0 + k), dg[a], P.sg);
      }
    }
    return;
  }
  // (with walls this group is away from them: no row wraps, and for the cavity
  // no column wraps either)
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const int xl = x0 == 0 ? nx - 4 : x0 - 4, xr = x0 + 4 == nx ? 0 : x0 + 4;
  const int64_t rows[3] = {(int64_t)ym * P.pitch, (int64_t)y * P.pitch, (int64_t)yp * P.pitch};
  // own groups of the 18 planes, and the one element node x0 (x0 + 3) takes
  // from the left (right) group of the x-shifted planes
  uint2 fo[9], go[9];
  float fe[9], ge[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const int64_t ro = rows[1 - EY[a]];
    fo[a] = ld_quad(fin + a * pl + ro + x0);
    go[a] = ld_quad(gin + a * pl + ro + x0);
    if (EX[a] == 1) {
      fe[a] = elem<S>(ld_quad(fin + a * pl + ro + xl), 3);
      ge[a] = elem<S>(ld_quad(gin + a * pl + ro + xl), 3);
    } else if (EX[a] == -1) {
      fe[a] = elem<S>(ld_quad(fin + a * pl + ro + xr), 0);
      ge[a] = elem<S>(ld_quad(gin + a * pl + ro + xr), 0);
    } else {
      fe[a] = ge[a] = 0.0f;
    }
  }
  unsigned fw[9][2], gw[9][2];  // packed results: [plane][low / high word]
  float fp[9], gp[9];           // results of the even node, until its odd neighbour is done
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float df[9], dg[9];  // in storage units (scaled deviations)
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      // node x0 + k pulls element k - e_ax of the own group (or the neighbour's)
      const int e = k - EX[a];
      df[a] = e < 0 || e > 3 ? fe[a] : elem<S>(fo[a], e);
      dg[a] = e < 0 || e > 3 ? ge[a] : elem<S>(go[a], e);
    }
    collide_scaled(P, df, dg);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      if (k & 1) {
        fw[a][k >> 1] = pack2<S>(fp[a], df[a]);
        gw[a][k >> 1] = pack2<S>(gp[a], dg[a]);
      } else {
        fp[a] = df[a];
        gp[a] = dg[a];
      }
    }
  }
  const int64_t own = (int64_t)y * P.pitch + x0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    __stcs(reinterpret_cast<uint2*>(fout + a * pl + own), make_uint2(fw[a][0], fw[a][1]));
    __stcs(reinterpret_cast<uint2*>(gout + a * pl + own), make_uint2(gw[a][0], gw[a][1]));
  }
}

namespace {
template <typename S, int BC>
cudaError_t go(const Launch& L, const void* fin, const void* gin, void* fout, void* gout,
               const DevStatus* st) {
  const dim3 b = L.block;
  const dim3 g((L.P.nx / 2 + b.x - 1) / b.x, (L.P.ny + b.y - 1) / b.y);
  k_step_pair<S, BC><<<g, b, 0, L.stream>>>(L.P, (const S*)fin, (const S*)gin, (S*)fout,
                                            (S*)gout, st);
  return cudaGetLastError();
}
template <typename S>
cudaError_t go_bc(const Launch& L, const void* fin, const void* gin, void* fout, void* gout,
                  const DevStatus* st) {
  switch (L.P_bc) {
    case BC_PERIODIC: return go<S, BC_PERIODIC>(L, fin, gin, fout, gout, st);
    case BC_CAVITY: return go<S, BC_CAVITY>(L, fin, gin, fout, gout, st);
    default: return go<S, BC_CHANNEL>(L, fin, gin, fout, gout, st);
  }
}
}  // namespace

// (whole lattices only: a y-slab context steps node by node)
bool quad_step_eligible(const Launch& L) {
  return !L.force && L.P.smodel < 2 && L.storage != 0 && L.P.nx % 4 == 0 && L.P.y0 == 0 &&
         L.P.y1 == L.P.ny;
}

namespace {
template <typename S, int BC>
cudaError_t go_quad(const Launch& L, const void* fin, const void* gin, void* fout, void* gout,
                    const DevStatus* st) {
  const dim3 b(128, 1);
  const dim3 g((L.P.nx / 4 + b.x - 1) / b.x, L.P.ny);
  k_step_quad<S, BC><<<g, b, 0, L.stream>>>(L.P, (const S*)fin, (const S*)gin, (S*)fout,
                                            (S*)gout, st);
  return cudaGetLastError();
}
template <typename S>
cudaError_t go_quad_bc(const Launch& L, const void* fin, const void* gin, void* fout,
                       void* gout, const DevStatus* st) {
  switch (L.P_bc) {
    case BC_PERIODIC: return go_quad<S, BC_PERIODIC>(L, fin, gin, fout, gout, st);
    case BC_CAVITY: return go_quad<S, BC_CAVITY>(L, fin, gin, fout, gout, st);
    default: return go_quad<S, BC_CHANNEL>(L, fin, gin, fout, gout, st);
  }
}
}  // namespace

cudaError_t launch_step_quad(const Launch& L, const void* fin, const void* gin, void* fout,
                             void* gout, const DevStatus* st) {
  if (L.storage == 1) return go_quad_bc<__half>(L, fin, gin, fout, gout, st);
  return go_quad_bc<__nv_bfloat16>(L, fin, gin, fout, gout, st);
}

bool pair_step_eligible(const Launch& L) {
  return !L.force && L.P.smodel < 2 && L.storage != 0 && L.P.nx % 2 == 0 && L.P.y0 == 0 &&
         L.P.y1 == L.P.ny;
}

cudaError_t launch_step_pair(const Launch& L, const void* fin, const void* gin, void* fout,
                             void* gout, const DevStatus* st) {
  if (L.storage == 1) return go_bc<__half>(L, fin, gin, fout, gout, st);
  return go_bc<__nv_bfloat16>(L, fin, gin, fout, gout, st);
}

}  // namespace ddflb
