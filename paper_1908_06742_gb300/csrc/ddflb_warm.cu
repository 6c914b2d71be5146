// Warm-start initial fields from a surrogate prediction, on the device.
//
// The learned warm start predicts the steady cavity fields; the prediction only
// initialises the populations (equilibrium plus the Chapman-Enskog
// non-equilibrium part of Secs. 2 and 3, written by ddflb_init from the fields
// and gradients produced here).  One thread per node reads the network output
// (NHWC, FP32) and writes rho, u, phi and the six gradient planes:
//   u = U p0, U p1;  phi = clamp(p2, lo, hi);  rho = 1 + U^2 p4;
//   omega = p3 * scale * U / n (the network's normalised vorticity);
//   d_x, d_y of u and phi: central differences inside, one-sided differences
//   on the first and last row and column;
//   the off-diagonal pair splits into the symmetric part of the differences
//   and the predicted vorticity: d_x u_y = S_xy + omega/2, d_y u_x = S_xy - omega/2.
// Each product and sum is rounded once in a fixed order (explicit _rn
// intrinsics, no contraction), so the result is reproducible bit for bit.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/ddflb.h"
#include "ddflb_internal.h"

namespace ddflb {
namespace {

struct WarmArgs {
  const float* pred;
  int nx, ny, cs;
  float u, oscale, n, lo, hi;
  float *rho, *ux, *uy, *phi, *grads;
};

__device__ __forceinline__ float chan(const WarmArgs& A, int x, int y, int c) {
  return A.pred[((int64_t)y * A.nx + x) * A.cs + c];
}

__device__ __forceinline__ float phi_at(const WarmArgs& A, int x, int y) {
  return fminf(fmaxf(chan(A, x, y, 2), A.lo), A.hi);
}

// derivative along one axis from the values at i - 1, i, i + 1 (m, c, p) of a
// line of length len: central inside, one-sided at the ends (unit spacing)
__device__ __forceinline__ float diff(float m, float c, float p, int i, int len) {
  if (len < 2) return 0.0f;
  if (i == 0) return __fsub_rn(p, c);
  if (i == len - 1) return __fsub_rn(c, m);
  return __fmul_rn(__fsub_rn(p, m), 0.5f);
}

__global__ void __launch_bounds__(256) k_warm(WarmArgs A) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= A.nx) return;
  const int xm = max(x - 1, 0), xp = min(x + 1, A.nx - 1);
  const int ym = max(y - 1, 0), yp = min(y + 1, A.ny - 1);
  const float U = A.u;
  auto vx = [&](int i, int j) { return __fmul_rn(chan(A, i, j, 0), U); };
  auto vy = [&](int i, int j) { return __fmul_rn(chan(A, i, j, 1), U); };
  const float ux = vx(x, y), uy = vy(x, y), ph = phi_at(A, x, y);
  const float dxux = diff(vx(xm, y), ux, vx(xp, y), x, A.nx);
  const float dyux = diff(vx(x, ym), ux, vx(x, yp), y, A.ny);
  const float dxuy = diff(vy(xm, y), uy, vy(xp, y), x, A.nx);
  const float dyuy = diff(vy(x, ym), uy, vy(x, yp), y, A.ny);
  const float dxph = diff(phi_at(A, xm, y), ph, phi_at(A, xp, y), x, A.nx);
  const float dyph = diff(phi_at(A, x, ym), ph, phi_at(A, x, yp), y, A.ny);
  const float om = __fdiv_rn(__fmul_rn(__fmul_rn(chan(A, x, y, 3), A.oscale), U), A.n);
  const float sxy = __fmul_rn(0.5f, __fadd_rn(dxuy, dyux));
  const float hom = __fmul_rn(0.5f, om);
  const int64_t o = (int64_t)y * A.nx + x, N = (int64_t)A.nx * A.ny;
  A.ux[o] = ux;
  A.uy[o] = uy;
  A.phi[o] = ph;
  A.rho[o] = __fadd_rn(1.0f, __fmul_rn(__fmul_rn(chan(A, x, y, 4), U), U));
  A.grads[o] = dxux;
  A.grads[N + o] = __fsub_rn(sxy, hom);
  A.grads[2 * N + o] = __fadd_rn(sxy, hom);
  A.grads[3 * N + o] = dyuy;
  A.grads[4 * N + o] = dxph;
  A.grads[5 * N + o] = dyph;
}

thread_local char g_warm_err[256];

}  // namespace
}  // namespace ddflb

using namespace ddflb;

extern "C" ddflb_status ddflb_warm_fields(const float* pred, int32_t nx, int32_t ny, int32_t cs,
                                          double u_lid, double omega_scale, double phi_lo,
                                          double phi_hi, float* rho, float* ux, float* uy,
                                          float* phi, float* grads, void* stream) {
  if (!pred || !rho || !ux || !uy || !phi || !grads) {
    set_error("warm_fields: NULL pointer");
    return DDFLB_EINVAL;
  }
  if (nx < 1 || ny < 1 || ny > 65535 || cs < 5 || !(u_lid > 0.0) || !(phi_lo <= phi_hi)) {
    snprintf(g_warm_err, sizeof g_warm_err,
             "warm_fields: need nx >= 1, 1 <= ny <= 65535, channel stride >= 5, u_lid > 0, phi_lo <= phi_hi "
             "(got %d x %d, cs %d, u %g, [%g, %g])", nx, ny, cs, u_lid, phi_lo, phi_hi);
    set_error(g_warm_err);
    return DDFLB_EINVAL;
  }
  WarmArgs A{pred, nx, ny, cs, (float)u_lid, (float)omega_scale, (float)nx, (float)phi_lo,
             (float)phi_hi, rho, ux, uy, phi, grads};
  k_warm<<<dim3((nx + 255) / 256, ny), 256, 0, (cudaStream_t)stream>>>(A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_warm_err, sizeof g_warm_err, "warm_fields: %s", cudaGetErrorString(e));
    set_error(g_warm_err);
    return DDFLB_ECUDA;
  }
  return DDFLB_OK;
}
