// Internal interface between the C ABI (ddflb_api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ddflb.h"
#include "ddflb_device.cuh"

namespace ddflb {

constexpr int kReduceThreads = 256;
constexpr int kReduceBlocks = 608;  // 4 per SM on a 152-SM GB300; fixed for deterministic sums

struct FieldPtrs {
  // 0..7: rho, ux, uy, phi, sxx, sxy, syy, omega; 8..17 (read only if derived):
  // dxux, dyux, dxuy, dyuy, dxphi, dyphi, Q, R, lamb_x, lamb_y (any may be null)
  float* p[18];
  int derived;
};

struct InitPtrs {
  const float *rho, *ux, *uy, *phi, *grads;
};

struct Launch {
  LbParams P;
  int P_bc;
  int storage;  // 0 fp32, 1 fp16, 2 bf16
  bool force;   // a body force acts (the FORCE kernel variants)
  dim3 block;
  cudaStream_t stream;
};

// y-slabs of one lattice on one device, for the single-launch halo exchange
constexpr int kMaxLocalSlabs = 64;
struct HaloSlab {
  void* buf;            // current population buffer (flow planes, then scalar)
  int64_t gofs_elems;   // elements from the flow planes to the scalar planes
  int64_t plane;        // elements per plane
  int y0, y1;           // own buffer rows [y0, y1)
};
struct HaloSlabs {
  HaloSlab s[kMaxLocalSlabs];
  int n, nx, pitch, periodic;
};

cudaError_t launch_halo_pack(const Launch& L, const void* buf, size_t gofs_bytes, void* down,
                             void* up);
cudaError_t launch_halo_unpack(const Launch& L, void* buf, size_t gofs_bytes,
                               const void* from_below, const void* from_above);
cudaError_t launch_halo_local(const HaloSlabs& H, int storage, cudaStream_t stream);

cudaError_t launch_step(const Launch& L, const void* fin, const void* gin, void* fout, void* gout,
                        const DevStatus* st);
cudaError_t launch_fields(const Launch& L, const void* fin, const void* gin, const FieldPtrs& out);
cudaError_t launch_pops(const Launch& L, const void* fin, const void* gin, float* f, float* g);
cudaError_t launch_init(const Launch& L, const InitPtrs& in, void* fout, void* gout);
cudaError_t launch_reduce(const Launch& L, const void* fin, const void* gin, float* uprev,
                          int mode, double* partials, DevStatus* st);

// Shared by the single-lattice and batched entry points (ddflb_api.cu).
void set_error(const char* msg);                     // thread-local ddflb_last_error()
LbParams make_lbparams(const ddflb_params* p, int pitch);

}  // namespace ddflb
