// Device building blocks of the fused DDF lattice Boltzmann step (sm_103a).
//
// Method: Hajabdollahi & Premnath, arXiv 1908.06742.
//   Sec. 2  flow MRT collision in the non-orthogonal basis (Eqs. basisvectors,
//           MRT-LBEfluidmotion_transformed, eqmrawmoment), F = 0
//   Sec. 3  scalar MRT collision with anisotropic third-order equilibria
//           (Eqs. MRT-LBECDE, eqmrawmoment_CDE)
//   Sec. 4  local strain rate and vorticity from non-equilibrium moments
//           (Eqs. crossderivativeRHS1/2, offdiagvelderivativeresult1/2,
//           diagvelderivativeresult1/2, vorticityexpression)
//   App. B  explicit inverse of the raw-moment basis (used for T^-1 below)
//
// Storage: populations live in structure-of-arrays planes [9][ny][pitch] per
// lattice, as deviations from the rest equilibrium times a per-lattice scale.
// All arithmetic here is FP32 on those deviations, which keeps the O(u) and
// O(u*k) signals far above the rounding of the O(1) rest part.
//
// Lattice velocities (Eq. particlevelocities), a = 0..8:
//   e_x = (0, 1, 0,-1, 0, 1,-1,-1, 1),  e_y = (0, 0, 1, 0,-1, 1, 1,-1,-1)
// Opposites: 1<->3, 2<->4, 5<->7, 6<->8.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace ddflb {

enum Bc : int { BC_PERIODIC = 0, BC_CAVITY = 1, BC_CHANNEL = 2 };

// Parameters of one lattice pair, passed by value to every kernel.
struct LbParams {
  int nx, ny, pitch;
  int64_t plane;          // elements per population plane (ny * pitch)
  float wf[9];            // flow relaxation rates, Eq. (relaxationtimematrix_fluidmotion)
  float wg[9];            // scalar relaxation rates, Eq. (relaxationtimematrix_CDE)
  float b1, b2;           // beta1, beta2
  float inv_db;           // 1 / (beta1 - beta2)
  float cs2, cs2p;        // c_s^2, c_sphi^2
  float rho0, phi0;       // rest state (storage offset)
  float phimin;
  float sf, isf, sg, isg; // storage scale and its inverse, per lattice
  float wrf[9], wrg[9];   // rest weights of each lattice
  float lid[9];           // moving-wall momentum term 2 w_a rho0 e_ax u_lid / c_s^2 (deviation form)
  float abb_lid[9];       // anti-bounce-back source 2 w^phi_a (phi_lid - phi0)
  float abb_wall[9];      // anti-bounce-back source 2 w^phi_a (phi_wall - phi0)
};

// Device status block (one per lattice pair), written by the reductions.
struct DevStatus {
  double mass_dev;    // sum of (rho - rho0) at the last reduction
  double scalar_dev;  // sum of (phi - phi0)
  double u2;          // sum |u|^2
  double du2;         // sum |u - u_prev|^2 (check reductions)
  double residual;    // sqrt(du2 / u2) of the last check
  int32_t diverged;   // set once a sum is non-finite
  int32_t has_residual;
  int64_t pad;
};

// ------------------------------------------------------------ storage codec
template <typename S> struct Codec;
template <> struct Codec<float> {
  static __device__ __forceinline__ float load(const float* p, float) { return __ldg(p); }
  static __device__ __forceinline__ void store(float* p, float v, float) { __stcs(p, v); }
};
template <> struct Codec<__half> {
  static __device__ __forceinline__ float load(const __half* p, float inv) {
    return __half2float(__ldg(p)) * inv;
  }
  static __device__ __forceinline__ void store(__half* p, float v, float s) {
    __stcs(reinterpret_cast<unsigned short*>(p), __half_as_ushort(__float2half_rn(v * s)));
  }
};
template <> struct Codec<__nv_bfloat16> {
  static __device__ __forceinline__ float load(const __nv_bfloat16* p, float inv) {
    return __bfloat162float(__ldg(p)) * inv;
  }
  static __device__ __forceinline__ void store(__nv_bfloat16* p, float v, float s) {
    __stcs(reinterpret_cast<unsigned short*>(p), __bfloat16_as_ushort(__float2bfloat16_rn(v * s)));
  }
};

// ------------------------------------------------------------ pull streaming
// Gathers the pre-collision deviations df, dg of node (x, y) from the
// post-collision planes of the previous step (pull form of the
// collide-and-stream update, Eqs. MRT-LBEfluidmotion, MRT-LBECDE).  A link whose
// upstream node lies beyond a wall takes the node's own post-collision value of
// the opposite direction (half-way bounce-back); the flow adds the moving-wall
// term, the scalar flips sign and adds 2 w (phi_w - phi0).
template <typename S, int BC>
__device__ __forceinline__ void pull(const LbParams& P, const S* __restrict__ fin,
                                     const S* __restrict__ gin, int x, int y, float df[9],
                                     float dg[9]) {
  const int nx = P.nx, ny = P.ny;
  const int64_t pl = P.plane;
  int xm = x - 1, xp = x + 1, ym = y - 1, yp = y + 1;
  bool sxm = false, sxp = false, sym = false, syp = false;  // source beyond a wall
  if (BC == BC_PERIODIC || BC == BC_CHANNEL) {
    if (xm < 0) xm += nx;
    if (xp >= nx) xp -= nx;
  } else {
    sxm = xm < 0;
    sxp = xp >= nx;
  }
  if (BC == BC_PERIODIC) {
    if (ym < 0) ym += ny;
    if (yp >= ny) yp -= ny;
  } else {
    sym = ym < 0;
    syp = yp >= ny;  // the moving lid
  }
  const int64_t r0 = (int64_t)y * P.pitch;
  const int64_t rm = (int64_t)ym * P.pitch;
  const int64_t rp = (int64_t)yp * P.pitch;
  const int64_t own = r0 + x;
  // source offsets of directions 0..8 (source = x - e_a)
  const int64_t src[9] = {own, r0 + xm, rm + x, r0 + xp, rp + x, rm + xm, rm + xp, rp + xp, rp + xm};
  // direction a's source is beyond a wall
  const bool solid[9] = {false, sxm, sym, sxp, syp, sxm || sym, sxp || sym, sxp || syp, sxm || syp};
  const bool lidl[9] = {false, false, false, false, syp, false, false, syp, syp};
  constexpr int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    if (BC == BC_PERIODIC) {
      df[a] = Codec<S>::load(fin + a * pl + src[a], P.isf);
      dg[a] = Codec<S>::load(gin + a * pl + src[a], P.isg);
    } else {
      const bool bb = solid[a];
      const int64_t off = bb ? (int64_t)opp[a] * pl + own : (int64_t)a * pl + src[a];
      float vf = Codec<S>::load(fin + off, P.isf);
      float vg = Codec<S>::load(gin + off, P.isg);
      if (bb) {
        const bool lid = lidl[a];
        vf += lid ? P.lid[a] : 0.0f;
        vg = (lid ? P.abb_lid[a] : P.abb_wall[a]) - vg;
      }
      df[a] = vf;
      dg[a] = vg;
    }
  }
}

// ------------------------------------------------------------ moments
// Raw moments of the deviations in the order of Eq. (basisvectors):
// (k0, kx, ky, kxx + kyy, kxx - kyy, kxy, kxxy, kxyy, kxxyy).
struct Mom {
  float k0, kx, ky, m3, m4, kxy, kxxy, kxyy, kxxyy;
};

__device__ __forceinline__ Mom moments(const float d[9]) {
  Mom m;
  const float s5 = d[5] + d[7], s6 = d[6] + d[8];
  const float a5 = d[5] - d[7], a6 = d[6] - d[8];
  m.kxxyy = s5 + s6;
  m.kxy = s5 - s6;
  m.kxxy = a5 + a6;
  m.kxyy = a5 - a6;
  const float dx = d[1] - d[3], dy = d[2] - d[4];
  m.kx = dx + m.kxyy;
  m.ky = dy + m.kxxy;
  const float kxx = d[1] + d[3] + m.kxxyy;
  const float kyy = d[2] + d[4] + m.kxxyy;
  m.m3 = kxx + kyy;
  m.m4 = kxx - kyy;
  m.k0 = d[0] + (d[1] + d[2]) + (d[3] + d[4]) + m.kxxyy;
  return m;
}

// Back to populations with the explicit inverse of App. B (kxx, kyy from
// m3 = kxx + kyy and m4 = kxx - kyy).
__device__ __forceinline__ void populations(const Mom& m, float d[9]) {
  const float kxx = 0.5f * (m.m3 + m.m4), kyy = 0.5f * (m.m3 - m.m4);
  d[0] = m.k0 - m.m3 + m.kxxyy;
  d[1] = 0.5f * (m.kx + kxx - m.kxyy - m.kxxyy);
  d[2] = 0.5f * (m.ky + kyy - m.kxxy - m.kxxyy);
  d[3] = 0.5f * (-m.kx + kxx + m.kxyy - m.kxxyy);
  d[4] = 0.5f * (-m.ky + kyy + m.kxxy - m.kxxyy);
  const float p = m.kxy + m.kxxyy, q = m.kxxy + m.kxyy;
  const float r = m.kxxyy - m.kxy, s = m.kxxy - m.kxyy;
  d[5] = 0.25f * (p + q);
  d[6] = 0.25f * (r + s);
  d[7] = 0.25f * (p - q);
  d[8] = 0.25f * (r - s);
}

// Equilibrium moments in deviation form (moment minus its rest value).
// Flow: Eq. (eqmrawmoment); scalar: Eq. (eqmrawmoment_CDE) with beta1, beta2.
struct Eq {
  float e1, e2, e3, e4, e5, e6, e7, e8;
};

__device__ __forceinline__ Eq eq_flow(const LbParams& P, float k0, float rho, float jx, float jy,
                                      float ux, float uy) {
  Eq e;
  const float c = P.cs2, uxx = ux * ux, uyy = uy * uy, usq = uxx + uyy;
  e.e1 = jx;
  e.e2 = jy;
  e.e3 = 2.0f * c * k0 + rho * usq;
  e.e4 = rho * (uxx - uyy);
  e.e5 = jx * uy;
  e.e6 = jy * (c + uxx);
  e.e7 = jx * (c + uyy);
  e.e8 = c * c * k0 + rho * (c * usq + uxx * uyy);
  return e;
}

__device__ __forceinline__ Eq eq_scalar(const LbParams& P, float n0, float phi, float ux, float uy) {
  Eq e;
  const float c = P.cs2p, uxx = ux * ux, uyy = uy * uy, usq = uxx + uyy;
  const float px = phi * ux, py = phi * uy;
  e.e1 = px;
  e.e2 = py;
  e.e3 = 2.0f * c * n0 + phi * usq;
  e.e4 = phi * (uxx - uyy);
  e.e5 = px * uy;
  e.e6 = py * (P.b1 * c + uxx);
  e.e7 = px * (P.b2 * c + uyy);
  e.e8 = c * c * n0 + phi * (c * usq + uxx * uyy);
  return e;
}

// Macroscopic state of a node (Eq. hydrodynamic_fields with F = 0; phi = sum g).
struct Macro {
  float rho, ux, uy, phi;
};

__device__ __forceinline__ Macro macro(const LbParams& P, const Mom& mf, const Mom& mg) {
  Macro q;
  q.rho = P.rho0 + mf.k0;
  const float inv = __frcp_rn(q.rho);
  q.ux = mf.kx * inv;
  q.uy = mf.ky * inv;
  q.phi = P.phi0 + mg.k0;
  return q;
}

// MRT relaxation in moment space, m* = m - Lambda (m - m^eq).
__device__ __forceinline__ void relax_flow(const LbParams& P, Mom& m, const Eq& e) {
  m.m3 -= P.wf[3] * (m.m3 - e.e3);
  m.m4 -= P.wf[4] * (m.m4 - e.e4);
  m.kxy -= P.wf[5] * (m.kxy - e.e5);
  m.kxxy -= P.wf[6] * (m.kxxy - e.e6);
  m.kxyy -= P.wf[7] * (m.kxyy - e.e7);
  m.kxxyy -= P.wf[8] * (m.kxxyy - e.e8);
}

__device__ __forceinline__ void relax_scalar(const LbParams& P, Mom& n, const Eq& e) {
  n.kx -= P.wg[1] * (n.kx - e.e1);
  n.ky -= P.wg[2] * (n.ky - e.e2);
  n.m3 -= P.wg[3] * (n.m3 - e.e3);
  n.m4 -= P.wg[4] * (n.m4 - e.e4);
  n.kxy -= P.wg[5] * (n.kxy - e.e5);
  n.kxxy -= P.wg[6] * (n.kxxy - e.e6);
  n.kxyy -= P.wg[7] * (n.kxyy - e.e7);
  n.kxxyy -= P.wg[8] * (n.kxxyy - e.e8);
}

// ------------------------------------------------------------ local kinematics
// Sec. 4: from the pre-collision non-equilibrium moments
//   m3' = m3 - m3^eq, m4' = m4 - m4^eq, m5' = kxy - rho ux uy       (flow)
//   n1' = eta_x - phi ux, n2' = eta_y - phi uy, n5' = eta_xy - phi ux uy (scalar)
// d_i phi = -(w_i^phi / cs2p) n_i';  N = -w5 m5' / (rho cs2);
// N^phi = -w5^phi n5' / (phi cs2p) - (b1 uy dxphi + b2 ux dyphi) / phi;
// dxuy = (N^phi - b2 N)/(b1 - b2), dyux = (b1 N - N^phi)/(b1 - b2),
// dxux = -(w3 m3' + w4 m4')/(4 cs2 rho), dyuy = -(w3 m3' - w4 m4')/(4 cs2 rho),
// omega_z = (2 N^phi - (b1 + b2) N)/(b1 - b2).
struct Kin {
  float sxx, sxy, syy, omega;
};

__device__ __forceinline__ Kin kinematics(const LbParams& P, const Mom& mf, const Mom& mg,
                                          const Macro& q, const Eq& ef, const Eq& eg) {
  Kin k;
  const float m3n = mf.m3 - ef.e3, m4n = mf.m4 - ef.e4, m5n = mf.kxy - ef.e5;
  const float n1n = mg.kx - eg.e1, n2n = mg.ky - eg.e2, n5n = mg.kxy - eg.e5;
  const float inv_cs2p = __frcp_rn(P.cs2p);
  const float dxphi = -P.wg[1] * inv_cs2p * n1n;
  const float dyphi = -P.wg[2] * inv_cs2p * n2n;
  const float irho = __frcp_rn(q.rho);
  const float N = -P.wf[5] * m5n * irho * __frcp_rn(P.cs2);
  const float diag = -0.25f * irho * __frcp_rn(P.cs2);
  k.sxx = diag * (P.wf[3] * m3n + P.wf[4] * m4n);
  k.syy = diag * (P.wf[3] * m3n - P.wf[4] * m4n);
  k.sxy = 0.5f * N;
  if (fabsf(q.phi) >= P.phimin) {
    const float iphi = __frcp_rn(q.phi);
    const float Nphi = (-P.wg[5] * n5n * inv_cs2p - (P.b1 * q.uy * dxphi + P.b2 * q.ux * dyphi)) * iphi;
    k.omega = (2.0f * Nphi - (P.b1 + P.b2) * N) * P.inv_db;
  } else {
    k.omega = __int_as_float(0x7fc00000);  // NaN: the relations need phi != 0
  }
  return k;
}

}  // namespace ddflb
