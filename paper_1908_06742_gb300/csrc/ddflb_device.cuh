// Device building blocks of the fused DDF lattice Boltzmann step (sm_103a).
//
// Method: Hajabdollahi & Premnath, arXiv 1908.06742.
//   Sec. 2  flow MRT collision in the non-orthogonal basis (Eqs. basisvectors,
//           MRT-LBEfluidmotion_transformed, eqmrawmoment), with the body-force
//           source moments when a force acts
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
  int nx, ny, pitch;      // ny: rows of the population buffers
  int y0, y1;             // buffer rows this context updates and reports, [y0, y1): all
                          // rows for a whole lattice; a y-slab's buffers add a ghost row
                          // on each face shared with another slab
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
  // body force (Sec. 2): F = (fx + field_x, fy + field_y) * fmod at every node
  float fx, fy, fmod;
  const float* ffield;    // optional [2][ny][nx] (row stride nx), or null
  int smodel;             // scalar collision: 0 MRT, 1 SRT (MRT with equal rates),
                          // 2 cascaded (App. C), 3 central moments (App. D)
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
// Loads take the read-only (non-coherent) path by default, for kernels that run
// one step per launch; COH = true reads through L2 only (ld.global.cg), for a
// persistent kernel whose planes are rewritten by other CTAs between its steps.
template <bool COH, typename T>
__device__ __forceinline__ T ld_pop(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
template <typename S> struct Codec;
template <> struct Codec<float> {
  template <bool COH = false>
  static __device__ __forceinline__ float load(const float* p, float) { return ld_pop<COH>(p); }
  static __device__ __forceinline__ void store(float* p, float v, float) { __stcs(p, v); }
};
template <> struct Codec<__half> {
  template <bool COH = false>
  static __device__ __forceinline__ float load(const __half* p, float inv) {
    return __half2float(ld_pop<COH>(p)) * inv;
  }
  static __device__ __forceinline__ void store(__half* p, float v, float s) {
    __stcs(reinterpret_cast<unsigned short*>(p), __half_as_ushort(__float2half_rn(v * s)));
  }
};
template <> struct Codec<__nv_bfloat16> {
  template <bool COH = false>
  static __device__ __forceinline__ float load(const __nv_bfloat16* p, float inv) {
    return __bfloat162float(ld_pop<COH>(p)) * inv;
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
template <typename S, int BC, bool COH = false>
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
  // in-plane offsets are 32-bit (a padded plane holds fewer than 2^32
  // elements); each plane's base pointer is the same for the whole warp
  const uint32_t pitch = (uint32_t)P.pitch;
  const uint32_t r0 = (uint32_t)y * pitch;
  const uint32_t rm = (uint32_t)ym * pitch;
  const uint32_t rp = (uint32_t)yp * pitch;
  const uint32_t own = r0 + (uint32_t)x;
  // source offsets of directions 0..8 (source = x - e_a); an offset whose
  // source lies beyond a wall is never used
  const uint32_t src[9] = {own,      r0 + xm, rm + x,  r0 + xp, rp + x,
                           rm + xm,  rm + xp, rp + xp, rp + xm};
  // direction a's source is beyond a wall
  const bool solid[9] = {false, sxm, sym, sxp, syp, sxm || sym, sxp || sym, sxp || syp, sxm || syp};
  const bool lidl[9] = {false, false, false, false, syp, false, false, syp, syp};
  constexpr int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    if (BC == BC_PERIODIC) {
      df[a] = Codec<S>::template load<COH>(fin + a * pl + src[a], P.isf);
      dg[a] = Codec<S>::template load<COH>(gin + a * pl + src[a], P.isg);
    } else {
      const bool bb = solid[a];
      const int64_t po = (int64_t)(bb ? opp[a] : a) * pl;
      const uint32_t off = bb ? own : src[a];
      float vf = Codec<S>::template load<COH>(fin + po + off, P.isf);
      float vg = Codec<S>::template load<COH>(gin + po + off, P.isg);
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
// Raw moments of the deviations in the basis of Eq. (basisvectors), with the
// two even moments that carry the rest state taken relative to it:
//   m3h = (kxx + kyy) - 2 c k0,  m8h = kxxyy - c^2 k0   (c = c_s^2 = 1/3),
// which are exactly the parts the rest-state equilibrium does not cancel.
//
// Summation order is chosen per lattice so that the dominant parts cancel
// exactly before any rounding (Sterbenz: a - b is exact for b/2 <= a <= 2b):
//  - the flow deviations are dominated by the O(u) odd part, so opposite
//    directions are added first (f_a + f_abar is small and exact);
//  - the scalar deviations are dominated by w_a (phi - phi0), so equal-weight
//    directions are differenced first, and the rest-part combinations
//    sum_a d_a (|e_a|^2 - 2c) and sum_a d_a (e_ax^2 e_ay^2 - c^2) are formed
//    from differences against q = d_0 / 4 (w_0 / 4 = w_1 = 4 w_5 at c = 1/3).
struct Mom {
  float k0, kx, ky, m3h, m4, kxy, kxxy, kxyy, m8h;
};

__device__ __forceinline__ Mom moments_flow(const float d[9]) {
  Mom m;
  const float s57 = d[5] + d[7], s68 = d[6] + d[8];
  const float a57 = d[5] - d[7], a68 = d[6] - d[8];
  m.kxy = s57 - s68;
  m.kxxy = a57 + a68;
  m.kxyy = a57 - a68;
  m.kx = (d[1] - d[3]) + m.kxyy;
  m.ky = (d[2] - d[4]) + m.kxxy;
  const float s13 = d[1] + d[3], s24 = d[2] + d[4];
  m.m4 = s13 - s24;
  const float A = s13 + s24, B = s57 + s68;
  m.m3h = ((A + 4.0f * B) - 2.0f * d[0]) * (1.0f / 3.0f);
  m.m8h = ((8.0f * B - A) - d[0]) * (1.0f / 9.0f);
  m.k0 = d[0] + (A + B);
  return m;
}

__device__ __forceinline__ Mom moments_scalar(const float d[9]) {
  Mom m;
  const float a57 = d[5] - d[7], a68 = d[6] - d[8];
  m.kxy = (d[5] - d[6]) + (d[7] - d[8]);
  m.kxxy = a57 + a68;
  m.kxyy = a57 - a68;
  m.kx = (d[1] - d[3]) + m.kxyy;
  m.ky = (d[2] - d[4]) + m.kxxy;
  m.m4 = (d[1] - d[2]) + (d[3] - d[4]);
  const float q = 0.25f * d[0];
  const float t1 = ((d[1] - q) + (d[3] - q)) + ((d[2] - q) + (d[4] - q));
  const float t2 = ((4.0f * d[5] - q) + (4.0f * d[7] - q)) + ((4.0f * d[6] - q) + (4.0f * d[8] - q));
  m.m3h = (t1 + t2) * (1.0f / 3.0f);
  const float u5 = (8.0f * d[5] - q) - d[1], u6 = (8.0f * d[6] - q) - d[2];
  const float u7 = (8.0f * d[7] - q) - d[3], u8 = (8.0f * d[8] - q) - d[4];
  m.m8h = ((u5 + u7) + (u6 + u8)) * (1.0f / 9.0f);
  m.k0 = d[0] + ((d[1] + d[3]) + (d[2] + d[4])) + ((d[5] + d[7]) + (d[6] + d[8]));
  return m;
}

// Populations from raw moments (deviation form, m3 = kxx + kyy and
// m8 = kxxyy in full) with the explicit inverse of App. B.
__device__ __forceinline__ void populations(float k0, float kx, float ky, float m3, float m4,
                                            float kxy, float kxxy, float kxyy, float kxxyy,
                                            float d[9]) {
  const float kxx = 0.5f * (m3 + m4), kyy = 0.5f * (m3 - m4);
  d[0] = k0 - m3 + kxxyy;
  d[1] = 0.5f * (kx + kxx - kxyy - kxxyy);
  d[2] = 0.5f * (ky + kyy - kxxy - kxxyy);
  d[3] = 0.5f * (-kx + kxx + kxyy - kxxyy);
  d[4] = 0.5f * (-ky + kyy + kxxy - kxxyy);
  const float p = kxy + kxxyy, q = kxxy + kxyy;
  const float r = kxxyy - kxy, s = kxxy - kxyy;
  d[5] = 0.25f * (p + q);
  d[6] = 0.25f * (r + s);
  d[7] = 0.25f * (p - q);
  d[8] = 0.25f * (r - s);
}

// Macroscopic state of a node (Eq. hydrodynamic_fields; phi = sum g).  Without
// a force u = j / rho; macro_force below adds the half-force shift first.
struct Macro {
  float rho, irho, ux, uy, phi;
};

__device__ __forceinline__ Macro macro(const LbParams& P, const Mom& mf, const Mom& mg) {
  Macro q;
  q.rho = P.rho0 + mf.k0;
  q.irho = __frcp_rn(q.rho);
  q.ux = mf.kx * q.irho;
  q.uy = mf.ky * q.irho;
  q.phi = P.phi0 + mg.k0;
  return q;
}

// Non-equilibrium moments m - m^eq (entries 1..8 of Eq. (basisvectors)); the
// equilibria are Eq. (eqmrawmoment) for the flow and Eq. (eqmrawmoment_CDE)
// for the scalar, written relative to the rest state like Mom (c = 1/3):
//   m3^eq - 2c k0 = rho |u|^2,  m8^eq - c^2 k0 = rho (c |u|^2 + ux^2 uy^2).
struct Neq {
  float n1, n2, n3, n4, n5, n6, n7, n8;
};

__device__ __forceinline__ Neq neq_flow(const Mom& m, const Macro& q) {
  Neq n;
  const float c = 1.0f / 3.0f;
  const float uxx = q.ux * q.ux, uyy = q.uy * q.uy, usq = uxx + uyy;
  n.n1 = 0.0f;  // momentum is conserved
  n.n2 = 0.0f;
  n.n3 = m.m3h - q.rho * usq;
  n.n4 = m.m4 - q.rho * (uxx - uyy);
  n.n5 = m.kxy - m.kx * q.uy;
  n.n6 = m.kxxy - m.ky * (c + uxx);
  n.n7 = m.kxyy - m.kx * (c + uyy);
  n.n8 = m.m8h - q.rho * (c * usq + uxx * uyy);
  return n;
}

__device__ __forceinline__ Neq neq_scalar(const LbParams& P, const Mom& g, const Mom& f,
                                          const Macro& q) {
  Neq n;
  const float c = 1.0f / 3.0f;
  const float uxx = q.ux * q.ux, uyy = q.uy * q.uy, usq = uxx + uyy;
  const float px = q.phi * q.ux, py = q.phi * q.uy;
  // first order: eta_x - phi u_x = (eta_x rho - phi j_x) / rho, with the product
  // phi j_x split exactly by an FMA so only the small result is rounded
  const float tx = q.phi * f.kx, ex = __fmaf_rn(q.phi, f.kx, -tx);
  const float ty = q.phi * f.ky, ey = __fmaf_rn(q.phi, f.ky, -ty);
  n.n1 = (__fmaf_rn(g.kx, q.rho, -tx) - ex) * q.irho;
  n.n2 = (__fmaf_rn(g.ky, q.rho, -ty) - ey) * q.irho;
  n.n3 = g.m3h - q.phi * usq;
  n.n4 = g.m4 - q.phi * (uxx - uyy);
  n.n5 = g.kxy - px * q.uy;
  n.n6 = g.kxxy - py * (P.b1 * c + uxx);
  n.n7 = g.kxyy - px * (P.b2 * c + uyy);
  n.n8 = g.m8h - q.phi * (c * usq + uxx * uyy);
  return n;
}

// Collision in increment form: f*_a = f_a - [T^-1 Lambda (m - m^eq)]_a
// (Eqs. MRT-LBEfluidmotion_transformed without force, MRT-LBECDE), so that only
// the small increment is built from moments and the stored value is rounded
// once.  w[] holds the relaxation rates of the lattice (w[0] = 0).
__device__ __forceinline__ void relax(const float w[9], const Neq& n, float d[9]) {
  const float d1 = w[1] * n.n1, d2 = w[2] * n.n2, d3 = w[3] * n.n3, d4 = w[4] * n.n4;
  const float d5 = w[5] * n.n5, d6 = w[6] * n.n6, d7 = w[7] * n.n7, d8 = w[8] * n.n8;
  const float dxx = 0.5f * (d3 + d4), dyy = 0.5f * (d3 - d4);
  d[0] -= d8 - d3;
  d[1] -= 0.5f * (d1 + dxx - d7 - d8);
  d[2] -= 0.5f * (d2 + dyy - d6 - d8);
  d[3] -= 0.5f * (-d1 + dxx + d7 - d8);
  d[4] -= 0.5f * (-d2 + dyy + d6 - d8);
  const float p = d5 + d8, q = d6 + d7, r = d8 - d5, s = d6 - d7;
  d[5] -= 0.25f * (p + q);
  d[6] -= 0.25f * (r + s);
  d[7] -= 0.25f * (p - q);
  d[8] -= 0.25f * (r - s);
}

// ------------------------------------------------------------ body force
// Sec. 2: the stored flow populations are f-bar = f - S/2, which makes the
// trapezoidal source explicit (Eq. MRT-LBEfluidmotion_transformed):
//   u = (sum f-bar e + F/2) / rho                      (Eq. hydrodynamic_fields)
//   m-bar* = m-bar - Lambda (m-bar - m^eq) + (I - Lambda/2) S
// with the source moments S of the force (the sigma' list after Eq. eqmrawmoment).
struct Force {
  float x, y;
};

__device__ __forceinline__ Force node_force(const LbParams& P, int x, int y) {
  float fx = P.fx, fy = P.fy;
  if (P.ffield != nullptr) {  // the field covers the context's own rows
    const int64_t c = (int64_t)(y - P.y0) * P.nx + x, n = (int64_t)P.nx * (P.y1 - P.y0);
    fx += P.ffield[c];
    fy += P.ffield[n + c];
  }
  return Force{fx * P.fmod, fy * P.fmod};
}

// Macroscopic state with the half-force velocity shift; the returned Mom has
// kx, ky replaced by rho u (what the equilibria and non-equilibria need).
__device__ __forceinline__ Macro macro_force(const LbParams& P, Mom& mf, const Mom& mg,
                                             const Force& F) {
  mf.kx += 0.5f * F.x;
  mf.ky += 0.5f * F.y;
  return macro(P, mf, mg);
}

struct Src {
  float s1, s2, s3, s4, s5, s6, s7, s8;
};

__device__ __forceinline__ Src source(const Force& F, const Macro& q) {
  Src s;
  const float sxx = 2.0f * F.x * q.ux, syy = 2.0f * F.y * q.uy;
  s.s1 = F.x;
  s.s2 = F.y;
  s.s3 = sxx + syy;
  s.s4 = sxx - syy;
  s.s5 = F.x * q.uy + F.y * q.ux;
  s.s6 = F.y * q.ux * q.ux + 2.0f * F.x * q.ux * q.uy;
  s.s7 = F.x * q.uy * q.uy + 2.0f * F.y * q.uy * q.ux;
  s.s8 = 2.0f * (F.x * q.ux * q.uy * q.uy + F.y * q.uy * q.ux * q.ux);
  return s;
}

// Forced collision increment: f-bar* = f-bar - T^-1 [Lambda n - (I - Lambda/2) S].
// With w1 = w2 = 0 the momentum gains exactly F (through d1, d2 = -F).
__device__ __forceinline__ void relax_source(const float w[9], const Neq& n, const Src& s,
                                             float d[9]) {
  const float d1 = w[1] * n.n1 - (1.0f - 0.5f * w[1]) * s.s1;
  const float d2 = w[2] * n.n2 - (1.0f - 0.5f * w[2]) * s.s2;
  const float d3 = w[3] * n.n3 - (1.0f - 0.5f * w[3]) * s.s3;
  const float d4 = w[4] * n.n4 - (1.0f - 0.5f * w[4]) * s.s4;
  const float d5 = w[5] * n.n5 - (1.0f - 0.5f * w[5]) * s.s5;
  const float d6 = w[6] * n.n6 - (1.0f - 0.5f * w[6]) * s.s6;
  const float d7 = w[7] * n.n7 - (1.0f - 0.5f * w[7]) * s.s7;
  const float d8 = w[8] * n.n8 - (1.0f - 0.5f * w[8]) * s.s8;
  const float dxx = 0.5f * (d3 + d4), dyy = 0.5f * (d3 - d4);
  d[0] -= d8 - d3;
  d[1] -= 0.5f * (d1 + dxx - d7 - d8);
  d[2] -= 0.5f * (d2 + dyy - d6 - d8);
  d[3] -= 0.5f * (-d1 + dxx + d7 - d8);
  d[4] -= 0.5f * (-d2 + dyy + d6 - d8);
  const float p = d5 + d8, q = d6 + d7, r = d8 - d5, s2 = d6 - d7;
  d[5] -= 0.25f * (p + q);
  d[6] -= 0.25f * (r + s2);
  d[7] -= 0.25f * (p - q);
  d[8] -= 0.25f * (r - s2);
}

// ------------------------------------------------------------ central-moment scalar models
// Non-equilibrium central moments nu = eta - eta^eq of the scalar lattice
// (Eq. centralmomentdefinitions_CDE, equilibria Eq. eqmcentralmoment_CDE),
// formed from the raw non-equilibrium moments n of neq_scalar by the binomial
// shift by u.  The raw image of the central equilibria equals the raw
// equilibria of Eq. (eqmrawmoment_CDE) up to third order; in the fourth-order
// moment it is larger by 2 c phi ((b2 - 1) ux^2 + (b1 - 1) uy^2).
struct CNeq {
  float x, y, xx, yy, xy, xxy, xyy, xxyy;
};

__device__ __forceinline__ CNeq central_neq(const LbParams& P, const Neq& n, const Macro& q) {
  const float c = 1.0f / 3.0f, ux = q.ux, uy = q.uy;
  const float rx = n.n1, ry = n.n2, rxx = 0.5f * (n.n3 + n.n4), ryy = 0.5f * (n.n3 - n.n4);
  const float rxy = n.n5, rxxy = n.n6, rxyy = n.n7;
  const float rxxyy = n.n8 - 2.0f * c * q.phi * ((P.b2 - 1.0f) * ux * ux + (P.b1 - 1.0f) * uy * uy);
  CNeq v;
  v.x = rx;
  v.y = ry;
  v.xx = rxx - 2.0f * ux * rx;
  v.yy = ryy - 2.0f * uy * ry;
  v.xy = rxy - uy * rx - ux * ry;
  v.xxy = rxxy - 2.0f * ux * rxy + ux * ux * ry - uy * rxx + 2.0f * ux * uy * rx;
  v.xyy = rxyy - 2.0f * uy * rxy + uy * uy * rx - ux * ryy + 2.0f * ux * uy * ry;
  v.xxyy = rxxyy - 2.0f * ux * rxyy - 2.0f * uy * rxxy + ux * ux * ryy + uy * uy * rxx +
           4.0f * ux * uy * rxy - 2.0f * ux * ux * uy * ry - 2.0f * ux * uy * uy * rx;
  return v;
}

// App. D (non-cascaded): each central moment relaxes at its own rate (xx + yy at
// w3, xx - yy at w4); the change is taken back to raw moments by the inverse
// binomial shift and to populations by the inverse of App. B, and added to d.
__device__ __forceinline__ void relax_central(const float w[9], const CNeq& v, const Macro& q,
                                              float d[9]) {
  const float ux = q.ux, uy = q.uy;
  const float Dx = -w[1] * v.x, Dy = -w[2] * v.y;
  const float Ds = -w[3] * (v.xx + v.yy), Dd = -w[4] * (v.xx - v.yy);
  const float Dxx = 0.5f * (Ds + Dd), Dyy = 0.5f * (Ds - Dd);
  const float Dxy = -w[5] * v.xy, Dxxy = -w[6] * v.xxy, Dxyy = -w[7] * v.xyy;
  const float Dxxyy = -w[8] * v.xxyy;
  const float Rxx = Dxx + 2.0f * ux * Dx, Ryy = Dyy + 2.0f * uy * Dy;
  const float Rxy = Dxy + uy * Dx + ux * Dy;
  const float Rxxy = Dxxy + 2.0f * ux * Dxy + ux * ux * Dy + uy * Dxx + 2.0f * ux * uy * Dx;
  const float Rxyy = Dxyy + 2.0f * uy * Dxy + uy * uy * Dx + ux * Dyy + 2.0f * ux * uy * Dy;
  const float Rxxyy = Dxxyy + 2.0f * ux * Dxyy + 2.0f * uy * Dxxy + ux * ux * Dyy + uy * uy * Dxx +
                      4.0f * ux * uy * Dxy + 2.0f * ux * ux * uy * Dy + 2.0f * ux * uy * uy * Dx;
  float dd[9];
  populations(0.0f, Dx, Dy, Rxx + Ryy, Rxx - Ryy, Rxy, Rxxy, Rxyy, Rxxyy, dd);
#pragma unroll
  for (int a = 0; a < 9; ++a) d[a] += dd[a];
}

// App. C (cascaded): the changes h1..h8 in the orthogonal basis K, found order by
// order so that every central moment relaxes at its rate; g~ = g + K h.  K6 and
// K7 are the orthogonal 2|e_y> - 3|e_x^2 e_y>, 2|e_x> - 3|e_x e_y^2> (the forms
// the paper's inner products and expansion of g~ require).
__device__ __forceinline__ void relax_cascaded(const float w[9], const CNeq& v, const Macro& q,
                                               float d[9]) {
  const float ux = q.ux, uy = q.uy, ux2 = ux * ux, uy2 = uy * uy;
  const float h1 = -w[1] * v.x * (1.0f / 6.0f);
  const float h2 = -w[2] * v.y * (1.0f / 6.0f);
  const float h3 = -w[3] * (v.xx + v.yy) * (1.0f / 12.0f) + (ux * h1 + uy * h2);
  const float h4 = -w[4] * (v.xx - v.yy) * 0.25f + 3.0f * (ux * h1 - uy * h2);
  const float h5 = -w[5] * v.xy * 0.25f + 1.5f * (ux * h2 + uy * h1);
  const float h6 = w[6] * v.xxy * 0.25f - 2.0f * ux * h5 - 0.5f * uy * h4 - 1.5f * uy * h3 +
                   (1.0f + 1.5f * ux2) * h2 + 3.0f * ux * uy * h1;
  const float h7 = w[7] * v.xyy * 0.25f - 2.0f * uy * h5 + 0.5f * ux * h4 - 1.5f * ux * h3 +
                   3.0f * ux * uy * h2 + (1.0f + 1.5f * uy2) * h1;
  const float h8 = -w[8] * v.xxyy * 0.25f - 2.0f * ux * h7 - 2.0f * uy * h6 -
                   4.0f * ux * uy * h5 + 0.5f * (ux2 - uy2) * h4 -
                   (2.0f + 1.5f * (ux2 + uy2)) * h3 + (2.0f + 3.0f * ux2) * uy * h2 +
                   (2.0f + 3.0f * uy2) * ux * h1;
  constexpr int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const float x = (float)ex[a], y = (float)ey[a], x2 = x * x, y2 = y * y;
    d[a] += x * h1 + y * h2 + (3.0f * (x2 + y2) - 4.0f) * h3 + (x2 - y2) * h4 + x * y * h5 +
            (2.0f * y - 3.0f * x2 * y) * h6 + (2.0f * x - 3.0f * x * y2) * h7 +
            (9.0f * x2 * y2 - 6.0f * (x2 + y2) + 4.0f) * h8;
  }
}

// Scalar collision of the model SM (0: the MRT of Sec. 3, also used for the
// SRT with equal rates; 2 cascaded; 3 central moments), given the scalar
// non-equilibrium moments ng.
template <int SM>
__device__ __forceinline__ void collide_scalar(const LbParams& P, const Neq& ng, const Macro& q,
                                               float dg[9]) {
  if (SM == 0) {
    relax(P.wg, ng, dg);
  } else {
    const CNeq v = central_neq(P, ng, q);
    if (SM == 2)
      relax_cascaded(P.wg, v, q, dg);
    else
      relax_central(P.wg, v, q, dg);
  }
}

// ------------------------------------------------------------ compensated odd moments
// The first- and third-order moments of both lattices are O(u) sums whose
// equilibria cancel them down to the small non-equilibrium part (flow n6, n7;
// scalar n1, n2, n6, n7, and the scalar xy moment), so the FP32 rounding of
// the O(u) partial sums, about one unit in the last place of a population per
// addition, lands in full on the non-equilibrium moments.  Accumulated over
// many steps it is as large as the rounding of the stored populations
// themselves.  With FP32 storage these moments are therefore formed with
// error-free transformations: every O(u) partial sum is kept as a value plus
// its exact rounding error (two-sum), the equilibrium's O(u) product is split
// exactly by an FMA, the leading parts cancel exactly (Sterbenz), and only the
// small remainder is rounded.  The relaxation (Eqs. MRT-LBEfluidmotion_transformed,
// MRT-LBECDE) and the kinematics of Sec. 4 are unchanged; only the rounding of
// the intermediate sums is removed.
struct Ef {
  float s, e;  // the unevaluated sum s + e
};

__device__ __forceinline__ Ef two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return Ef{s, (a - (s - bb)) + (b - bb)};
}

// a - k b for a constant k, with the product k b.s split exactly by an FMA
__device__ __forceinline__ float sub_scaled(const Ef& a, float k, const Ef& b) {
  const float p = k * b.s, pe = __fmaf_rn(k, b.s, -p);
  return (a.s - p) + ((a.e - pe) - k * b.e);
}

// ka a - kb b for constants ka, kb, both products split exactly by FMAs
__device__ __forceinline__ float cross_diff(float ka, const Ef& a, float kb, const Ef& b) {
  const float p = ka * a.s, pe = __fmaf_rn(ka, a.s, -p);
  const float r = kb * b.s, re = __fmaf_rn(kb, b.s, -r);
  return (p - r) + ((pe - re) + (ka * a.e - kb * b.e));
}

// j_x, j_y, k_xxy, k_xyy of one lattice's deviations (moments 1, 2, 6, 7 of
// Eq. basisvectors) as value + exact remainder
struct OddMom {
  Ef kx, ky, kxxy, kxyy;
};

__device__ __forceinline__ OddMom odd_moments(const float d[9]) {
  const Ef a57 = two_sum(d[5], -d[7]), a68 = two_sum(d[6], -d[8]);
  const Ef d13 = two_sum(d[1], -d[3]), d24 = two_sum(d[2], -d[4]);
  OddMom m;
  m.kxxy = two_sum(a57.s, a68.s);
  m.kxxy.e += a57.e + a68.e;
  m.kxyy = two_sum(a57.s, -a68.s);
  m.kxyy.e += a57.e - a68.e;
  m.kx = two_sum(d13.s, m.kxyy.s);
  m.kx.e += d13.e + m.kxyy.e;
  m.ky = two_sum(d24.s, m.kxxy.s);
  m.ky.e += d24.e + m.kxxy.e;
  return m;
}

// Replaces the O(u)-cancelling non-equilibrium moments of nf (n6, n7) and ng
// (n1, n2, n6, n7; n5 too if XY) by their compensated forms.  mf, mg, q are the
// plain moments and macroscopic state of the node; F the body force (zero
// without), whose half shifts the momentum as in macro_force.
template <bool XY>
__device__ __forceinline__ void neq_compensate(const LbParams& P, const float df[9],
                                               const float dg[9], const Mom& mf, const Mom& mg,
                                               const Macro& q, float hfx, float hfy, Neq& nf,
                                               Neq& ng) {
  const float c = 1.0f / 3.0f;
  OddMom of = odd_moments(df);
  const OddMom og = odd_moments(dg);
  if (hfx != 0.0f || hfy != 0.0f) {  // the half-force momentum shift, exactly
    const Ef sx = two_sum(of.kx.s, hfx), sy = two_sum(of.ky.s, hfy);
    of.kx = Ef{sx.s, sx.e + of.kx.e};
    of.ky = Ef{sy.s, sy.e + of.ky.e};
  }
  const float uxx = q.ux * q.ux, uyy = q.uy * q.uy;
  // flow: k_xxy - j_y (c + ux^2), k_xyy - j_x (c + uy^2)
  nf.n6 = sub_scaled(of.kxxy, c, of.ky) - mf.ky * uxx;
  nf.n7 = sub_scaled(of.kxyy, c, of.kx) - mf.kx * uyy;
  // scalar first order: eta_x - phi u_x = (eta_x rho - phi j_x) / rho, written
  // as ((rho0 eta_x - phi0 j_x) + eta_x (rho - rho0) - (phi - phi0) j_x) / rho,
  // whose leading parts rho0 eta_x and phi0 j_x cancel
  const float drho = mf.k0, dphi = mg.k0;
  const float n1 = (cross_diff(P.rho0, og.kx, P.phi0, of.kx) +
                    (og.kx.s * drho - dphi * of.kx.s)) * q.irho;
  const float n2 = (cross_diff(P.rho0, og.ky, P.phi0, of.ky) +
                    (og.ky.s * drho - dphi * of.ky.s)) * q.irho;
  ng.n1 = n1;
  ng.n2 = n2;
  // scalar third order: eta_xxy - phi u_y (b1 c + ux^2) with phi u_y = eta_y - n2
  const float b1c = P.b1 * c, b2c = P.b2 * c;
  const float px = og.kx.s - n1, py = og.ky.s - n2;
  ng.n6 = sub_scaled(og.kxxy, b1c, og.ky) + b1c * n2 - py * uxx;
  ng.n7 = sub_scaled(og.kxyy, b2c, og.kx) + b2c * n1 - px * uyy;
  if (XY) {  // eta_xy - phi ux uy, from two exact pair differences
    const Ef a56 = two_sum(dg[5], -dg[6]), a78 = two_sum(dg[7], -dg[8]);
    ng.n5 = ((a56.s + a78.s) + (a56.e + a78.e)) - px * q.uy;
  }
}

// Moments, macroscopic state and both collisions of one node, in place on the
// pulled deviations df, dg.  FORCE = false is the unforced step.  COMP: the
// odd non-equilibrium moments are compensated (FP32 storage).
template <bool FORCE, int SM = 0, bool COMP = false>
__device__ __forceinline__ void collide(const LbParams& P, int x, int y, float df[9],
                                        float dg[9]) {
  Mom mf = moments_flow(df);
  const Mom mg = moments_scalar(dg);
  if (FORCE) {
    const Force F = node_force(P, x, y);
    const Macro q = macro_force(P, mf, mg, F);
    Neq nf = neq_flow(mf, q), ng = neq_scalar(P, mg, mf, q);
    if (COMP) neq_compensate<false>(P, df, dg, mf, mg, q, 0.5f * F.x, 0.5f * F.y, nf, ng);
    relax_source(P.wf, nf, source(F, q), df);
    collide_scalar<SM>(P, ng, q, dg);
  } else {
    const Macro q = macro(P, mf, mg);
    Neq nf = neq_flow(mf, q), ng = neq_scalar(P, mg, mf, q);
    if (COMP) neq_compensate<false>(P, df, dg, mf, mg, q, 0.0f, 0.0f, nf, ng);
    relax(P.wf, nf, df);
    collide_scalar<SM>(P, ng, q, dg);
  }
}

// The unforced MRT collision of one node on populations held in storage units
// (the deviations times the power-of-two storage scales sf, sg of the 16-bit
// formats), without converting each population: the moments are linear, so
// those of the scaled populations are the scaled moments; only the density and
// momentum are brought back to physical units for rho and u, and the
// equilibrium products take sf rho (flow) and sg phi (scalar) in place of rho
// and phi.  Scaling by a power of two commutes with rounding (every sum,
// product and fused multiply-add of scaled operands rounds to exactly the
// scaled result), so this is bit-identical to collide<false, 0> on d / s
// followed by the storage conversion of d s, with 6 multiplies instead of 36.
__device__ __forceinline__ void collide_scaled(const LbParams& P, float df[9], float dg[9]) {
  const Mom mf = moments_flow(df), mg = moments_scalar(dg);
  Mom fu = mf;  // flow moments in physical units where the scalar lattice needs them
  fu.k0 = mf.k0 * P.isf;
  fu.kx = mf.kx * P.isf;
  fu.ky = mf.ky * P.isf;
  Mom gu = mg;
  gu.k0 = mg.k0 * P.isg;
  const Macro q = macro(P, fu, gu);
  Macro qf = q, qg = q;
  qf.rho = q.rho * P.sf;
  qg.phi = q.phi * P.sg;
  relax(P.wf, neq_flow(mf, qf), df);
  relax(P.wg, neq_scalar(P, mg, fu, qg), dg);
}

// Macroscopic state and the non-equilibrium moments the kinematics use.  With
// a force the flow moments are those of f = f-bar + S/2 (the distribution whose
// non-equilibrium part Sec. 4 relates to the velocity gradients).  The odd
// non-equilibrium moments (and the scalar xy moment) are compensated.
template <bool FORCE>
__device__ __forceinline__ Macro state(const LbParams& P, int x, int y, const float df[9],
                                       const float dg[9], Neq& nf, Neq& ng) {
  Mom mf = moments_flow(df);
  const Mom mg = moments_scalar(dg);
  Macro q;
  float hfx = 0.0f, hfy = 0.0f;
  Src s{};
  if (FORCE) {
    const Force F = node_force(P, x, y);
    hfx = 0.5f * F.x;
    hfy = 0.5f * F.y;
    q = macro_force(P, mf, mg, F);
    s = source(F, q);
  } else {
    q = macro(P, mf, mg);
  }
  nf = neq_flow(mf, q);
  ng = neq_scalar(P, mg, mf, q);
  neq_compensate<true>(P, df, dg, mf, mg, q, hfx, hfy, nf, ng);
  if (FORCE) {
    nf.n3 += 0.5f * s.s3;
    nf.n4 += 0.5f * s.s4;
    nf.n5 += 0.5f * s.s5;
    nf.n6 += 0.5f * s.s6;
    nf.n7 += 0.5f * s.s7;
    nf.n8 += 0.5f * s.s8;
  }
  return q;
}

// ------------------------------------------------------------ local kinematics
// Sec. 4, from the pre-collision non-equilibrium moments (nf: flow, ng: scalar):
//   d_i phi = -(w_i^phi / c_phi) ng_i;   N = -w5 nf_5 / (rho c);
//   N^phi = -w5^phi ng_5 / (phi c_phi) - (b1 uy dxphi + b2 ux dyphi) / phi;
//   dxux = -(w3 nf_3 + w4 nf_4) / (4 c rho),  dyuy = -(w3 nf_3 - w4 nf_4) / (4 c rho);
//   omega_z = (2 N^phi - (b1 + b2) N) / (b1 - b2);  S_xy = N / 2.
struct Kin {
  float sxx, sxy, syy, omega;
  float div;           // d_x u_x + d_y u_y = -w3 nf_3 / (2 c rho), formed without cancellation
  float dyux, dxuy;    // Eqs. (offdiagvelderivativeresult1), (offdiagvelderivativeresult2)
  float dxphi, dyphi;  // scalar gradient from the first-order non-equilibrium moments
};

__device__ __forceinline__ Kin kinematics(const LbParams& P, const Neq& nf, const Neq& ng,
                                          const Macro& q) {
  Kin k;
  const float inv_c = 3.0f;  // 1 / c_s^2 = 1 / c_sphi^2
  const float dxphi = -P.wg[1] * inv_c * ng.n1;
  const float dyphi = -P.wg[2] * inv_c * ng.n2;
  const float N = -P.wf[5] * nf.n5 * q.irho * inv_c;
  const float diag = -0.25f * q.irho * inv_c;
  k.sxx = diag * (P.wf[3] * nf.n3 + P.wf[4] * nf.n4);
  k.syy = diag * (P.wf[3] * nf.n3 - P.wf[4] * nf.n4);
  k.sxy = 0.5f * N;
  k.div = 2.0f * diag * P.wf[3] * nf.n3;
  k.dxphi = dxphi;
  k.dyphi = dyphi;
  if (fabsf(q.phi) >= P.phimin) {
    const float iphi = __frcp_rn(q.phi);
    // central-moment models: the central xy moment (equilibrium zero) and
    // (beta - 1) in the scalar-gradient correction
    const bool cm = P.smodel >= 2;
    const float n5 = cm ? ng.n5 - q.uy * ng.n1 - q.ux * ng.n2 : ng.n5;
    const float c1 = cm ? P.b1 - 1.0f : P.b1, c2 = cm ? P.b2 - 1.0f : P.b2;
    const float Nphi = (-P.wg[5] * n5 * inv_c - (c1 * q.uy * dxphi + c2 * q.ux * dyphi)) * iphi;
    k.omega = (2.0f * Nphi - (P.b1 + P.b2) * N) * P.inv_db;
    k.dxuy = (Nphi - P.b2 * N) * P.inv_db;
    k.dyux = (P.b1 * N - Nphi) * P.inv_db;
  } else {
    k.omega = __int_as_float(0x7fc00000);  // NaN: the relations need phi != 0
    k.dxuy = k.omega;
    k.dyux = k.omega;
  }
  return k;
}

// Invariants built from the local velocity gradient (the vortex-identification
// quantities named in Sec. 1), for a planar flow (omega along z, S in the
// x-y plane, so the omega_i omega_j S_ij term of R vanishes):
//   Q = -S_ij S_ij / 2 + omega^2 / 4,  R = S_ij S_jk S_ki / 3,
//   Lamb vector L = omega x u = (-omega u_y, omega u_x).
// For the 2x2 strain, S_ij S_jk S_ki = tr S (sxx^2 - sxx syy + syy^2 + 3 sxy^2):
// R is proportional to the divergence, which is small in a nearly incompressible
// flow, so it is formed from tr S directly (one moment, n_3) rather than as the
// difference sxx^3 + syy^3 of two nearly opposite cubes.
struct Inv {
  float q, r, lx, ly;
};

__device__ __forceinline__ Inv invariants(const Kin& k, const Macro& m) {
  Inv v;
  const float ss = k.sxx * k.sxx + k.syy * k.syy + 2.0f * k.sxy * k.sxy;
  v.q = -0.5f * ss + 0.25f * k.omega * k.omega;
  v.r = k.div * (k.sxx * k.sxx - k.sxx * k.syy + k.syy * k.syy + 3.0f * k.sxy * k.sxy) *
        (1.0f / 3.0f);
  v.lx = -k.omega * m.uy;
  v.ly = k.omega * m.ux;
  return v;
}

}  // namespace ddflb
