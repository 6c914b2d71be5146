// Kernels of the warm-start surrogate network (a small U-Net): BF16 tensor-core
// GEMM with FP32 accumulation and a fused bias + activation epilogue, plus the
// data-movement kernels that turn 3x3 convolutions into GEMMs (im2col in two
// layouts, col2im), pooling, upsampling, the activation derivative, bias
// gradients, the MSE loss and Adam.
//
// Tensors are NHWC with an explicit channel stride ("cs"), so a concatenation
// is two producers writing disjoint channel slices of one buffer.
//
// GEMM convention: C[M][N] = A[M][K] . B[N][K]^T (both operands K-contiguous,
// row-major), i.e. a convolution forward pass is C = im2col(X) . W^T with
// W[Cout][3][3][Cin].
#include <cuda.h>  // CUtensorMap and its enums (types only; the encoder is looked up at run time)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>

#include "../../include/ddflb.h"
#include "ddflb_internal.h"

namespace ddflb {
namespace nn {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ float act_fwd(float z, int act) {
  return act == 1 ? (z > 0.f ? z : 0.02f * z) : z;  // 1: leaky ReLU, slope 0.02
}

// ------------------------------------------------------------------ GEMM
// 128 x 128 CTA tile, K step 32, 8 warps (2 along M x 4 along N), each warp a
// 64 x 32 tile of m16n8k16 MMAs; operands staged in padded shared memory by
// cp.async with a two-stage pipeline.
constexpr int BM = 128, BN = 128, BK = 32, LDS = BK + 8;  // +8 bf16: conflict-free ldmatrix

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = pred ? 16 : 0;  // src-size 0: zero fill
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n"); }

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3,
                                        const void* p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(s));
}

__device__ __forceinline__ void mma16816(float c[4], const unsigned a[4], const unsigned b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct GemmArgs {
  const bf16* A;
  const bf16* B;
  int M, N, K, lda, ldb;
  float* Cf;   // optional FP32 output [M][ldc]
  bf16* Cb;    // optional BF16 output [M][ldcb]
  int ldc, ldcb;
  const float* bias;  // optional [N]
  int act;
  int accumulate;  // Cf += result (FP32 only)
  int kchunk;      // K range per blockIdx.z (split-K); == K when not split
  float* partial;  // split-K: slice z written to partial + z*M*N (row-major [M][N])
  // implicit 3x3 convolution (conv_c > 0): A is the NHWC activation seen
  // through a 4-D tensor map, row m of the product = pixel m, and k-step kt
  // reads tap kt / (conv_c / 64) (dy = tap / 3 - 1, dx = tap % 3 - 1) of the
  // 64-channel chunk kt % (conv_c / 64); a tile of 128 pixels is one box of
  // conv_bw x conv_bh x conv_bb (w, h, image)
  int conv_c, conv_w, conv_h;
  int conv_bw, conv_bh, conv_bb;
  // band mode (W a multiple of 128, tiles = 128-pixel row segments): the A map
  // reads bands of 130 pixels (the segment and one halo pixel each side) of one
  // input row; conv_ag = band-group slots (one group = the bands of all
  // channel chunks of one input row), conv_bs = slots of the B ring, or 0 when
  // the whole weight matrix stays resident in shared memory (N <= BN)
  int conv_ag, conv_bs;
};

__global__ void __launch_bounds__(256) k_gemm(GemmArgs g) {
  __shared__ __align__(16) bf16 sA[2][BM * LDS];
  __shared__ __align__(16) bf16 sB[2][BN * LDS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
  float acc[4][4][4] = {};
  const int kbeg = blockIdx.z * g.kchunk, kend = min(g.K, kbeg + g.kchunk);

  // each thread moves 2 x 16 B of A and of B per K step (128 rows x 4 chunks)
  auto load = [&](int stage, int k0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int idx = tid + r * 256, row = idx >> 2, ch = (idx & 3) * 8;
      const int gm = m0 + row, gk = k0 + ch;
      const bool pa = gm < g.M && gk < kend;
      cp_async16(&sA[stage][row * LDS + ch], pa ? g.A + (size_t)gm * g.lda + gk : g.A, pa);
      const int gn = n0 + row;
      const bool pb = gn < g.N && gk < kend;
      cp_async16(&sB[stage][row * LDS + ch], pb ? g.B + (size_t)gn * g.ldb + gk : g.B, pb);
    }
    cp_async_commit();
  };

  const int nk = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  if (nk > 0) load(0, kbeg);
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1;
    cp_async_wait0();
    __syncthreads();
    if (kt + 1 < nk) load(st ^ 1, kbeg + (kt + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned af[4][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = wm + i * 16 + (lane & 15), col = kk + (lane >> 4) * 8;
        ldsm_x4(af[i][0], af[i][1], af[i][2], af[i][3], &sA[st][row * LDS + col]);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        // two n8 tiles per ldmatrix.x4: rows n = wn + j*16 + (lane & 7) + ((lane >> 4) << 3)
        const int row = wn + j * 16 + (lane & 7) + ((lane >> 4) << 3);
        const int col = kk + ((lane >> 3) & 1) * 8;
        unsigned r0, r1, r2, r3;
        ldsm_x4(r0, r1, r2, r3, &sB[st][row * LDS + col]);
        bfr[2 * j][0] = r0;
        bfr[2 * j][1] = r1;
        bfr[2 * j + 1][0] = r2;
        bfr[2 * j + 1][1] = r3;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }
  // epilogue: c0,c1 at (lane/4, 2(lane%4) + {0,1}); c2,c3 eight rows below
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = m0 + wm + i * 16 + (lane >> 2) + h * 8;
        const int c = n0 + wn + j * 8 + (lane & 3) * 2;
        if (r >= g.M) continue;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (c + e >= g.N) continue;
          float v = acc[i][j][2 * h + e];
          if (g.partial) {
            g.partial[((size_t)blockIdx.z * g.M + r) * g.N + c + e] = v;
            continue;
          }
          if (g.bias) v += g.bias[c + e];
          v = act_fwd(v, g.act);
          if (g.Cf) {
            float* p = g.Cf + (size_t)r * g.ldc + c + e;
            *p = g.accumulate ? *p + v : v;
          }
          if (g.Cb) g.Cb[(size_t)r * g.ldcb + c + e] = __float2bfloat16_rn(v);
        }
      }
}

// ------------------------------------------------------------------ tcgen05 GEMM
// The same contraction on the 5th-generation tensor cores, warp-specialised,
// one CTA (4 warps) per 128 x BN tile of C (BN = 32, 64 or 128 from N):
//  - producer (warp 0, one thread): TMA (cp.async.bulk.tensor, 2-D tensor maps
//    over A [M][K] and B [N][K]) fills a ring of STAGES shared-memory slots,
//    one box of 64 K-elements (128 B) x rows per operand, written with the
//    128-byte swizzle: the canonical K-major SWIZZLE_128B layout, 8-row x 128-B
//    atoms of 1024 B stacked along M/N (stride byte offset 1024), the 16-byte
//    chunks of row r permuted by r mod 8; the K = 16 slices of a 64-wide step
//    start 32 B apart inside the atom.  The slot's `full` mbarrier counts the
//    bytes in (expect_tx); before refilling a slot the producer waits on its
//    `empty` mbarrier;
//  - MMA issuer (warp 1, one thread): waits on `full`, issues tcgen05.mma
//    (kind::f16, BF16 x BF16 -> FP32, M = 128, N = BN, K = 16 each) into an
//    accumulator in tensor memory (128 lanes x BN columns), tcgen05.commit
//    arrives on `empty` once those MMAs have read the slot, and on `done` after
//    the last;
//  - epilogue (all 4 warps): wait on `done`, read lanes 32w..32w+31 (rows of
//    C) with tcgen05.ld, add the bias, apply the activation, store.
// TMA zero-fills rows and K past the tensor edges.  Every mbarrier wait is
// bounded (globaltimer, 1 s): on expiry the CTA records an error
// (ddflb_nn_take_error), skips the epilogue, waits (bounded) for its copies in
// flight, frees its tensor memory and returns.
namespace tc {
constexpr int BM = 128, BK = 64;
constexpr int THREADS = 128;
template <int BN>
struct Cfg {
  static constexpr int STAGES = BN == 128 ? 4 : 6;
  static constexpr int A_TILE = BM * BK * 2, B_TILE = BN * BK * 2;  // bytes per slot
  static constexpr int STAGE = A_TILE + B_TILE;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 256;  // + alignment, barriers, slot
  static constexpr uint32_t COLS = BN < 32 ? 32 : BN;       // tensor-memory columns
  static constexpr uint32_t SBO = 1024;  // 8 rows x 128 B
  // instruction descriptor: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
  // both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};
}  // namespace tc

__device__ int g_tc_error;  // set (1) when a bounded wait of the tcgen05 GEMM ran out

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// shared-memory matrix descriptor for a K-major SWIZZLE_128B operand: start
// address >> 4 (bits 0-13), leading byte offset 16 B (unused for this layout,
// bits 16-29), stride byte offset >> 4 (bits 32-45), descriptor version 1
// (bits 46-47), layout type 2 = 128-byte swizzle (bits 61-63)
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait for the completion of the mbarrier phase with the given parity
// (the timer is read only once the phase is found incomplete)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t deadline = globaltimer_ns() + 1000000000ull;
  for (uint32_t it = 0; it < (1u << 24); ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 255 && globaltimer_ns() > deadline) return false;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// one 2-D TMA box (x = K element, y = row) into shared memory, counted on `bar`
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                       uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// one 4-D TMA box (c, w, h, image) into shared memory, counted on `bar`; the
// w and h coordinates may lie outside the image (the box reads zeros there)
__device__ __forceinline__ void tma_4d(uint32_t dst, const CUtensorMap* map, int c, int w, int h,
                                       int b, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(w), "r"(h), "r"(b), "r"(bar)
      : "memory");
}

#define DDFLB_R8(i) "=r"(r[i]), "=r"(r[i + 1]), "=r"(r[i + 2]), "=r"(r[i + 3]), \
                    "=r"(r[i + 4]), "=r"(r[i + 5]), "=r"(r[i + 6]), "=r"(r[i + 7])

// 32 consecutive FP32 columns of the calling thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t r[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : DDFLB_R8(0), DDFLB_R8(8), DDFLB_R8(16), DDFLB_R8(24)
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
#undef DDFLB_R8

// Epilogue of one accumulator row segment: 32 FP32 columns (cb .. cb+31) of
// row r, plus bias and activation, to the split-K partial buffer (slice z), the
// FP32 output (optionally accumulated) and/or the BF16 output; 16-byte stores
// where the layout allows (vf, vb).
__device__ __forceinline__ void store_row32(const GemmArgs& g, int r, int cb, int z,
                                            const uint32_t v[32], bool has_k, bool vf, bool vb) {
  float x[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    float t = has_k ? __uint_as_float(v[i]) : 0.0f;
    if (!g.partial) {
      if (g.bias && cb + i < g.N) t += g.bias[cb + i];
      t = act_fwd(t, g.act);
    }
    x[i] = t;
  }
  if (g.partial) {
    float* p = g.partial + ((size_t)z * g.M + r) * g.N;
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (cb + i < g.N) p[cb + i] = x[i];
    return;
  }
  const bool full_chunk = cb + 32 <= g.N;
  if (g.Cf) {
    float* p = g.Cf + (size_t)r * g.ldc + cb;
    if (vf && full_chunk) {
#pragma unroll
      for (int i = 0; i < 32; i += 4) {
        float4 o = make_float4(x[i], x[i + 1], x[i + 2], x[i + 3]);
        if (g.accumulate) {
          const float4 q = *reinterpret_cast<const float4*>(p + i);
          o.x += q.x; o.y += q.y; o.z += q.z; o.w += q.w;
        }
        *reinterpret_cast<float4*>(p + i) = o;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (cb + i < g.N) p[i] = g.accumulate ? p[i] + x[i] : x[i];
    }
  }
  if (g.Cb) {
    bf16* p = g.Cb + (size_t)r * g.ldcb + cb;
    if (vb && full_chunk) {
#pragma unroll
      for (int i = 0; i < 32; i += 8) {
        __align__(16) bf16 h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) h[e] = __float2bfloat16_rn(x[i + e]);
        *reinterpret_cast<uint4*>(p + i) = *reinterpret_cast<const uint4*>(h);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (cb + i < g.N) p[i] = __float2bfloat16_rn(x[i]);
    }
  }
}

template <int BN>
__global__ void __launch_bounds__(tc::THREADS) k_gemm_tc(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmB,
                                                         GemmArgs g) {
  using C = tc::Cfg<BN>;
  constexpr int S = C::STAGES;
  extern __shared__ uint8_t dsmem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // 1024-byte aligned ring of slots, then the mbarriers full[S], empty[S], done
  // and the tensor-memory address slot
  const uint32_t raw = smem_u32(dsmem);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint64_t* bars = reinterpret_cast<uint64_t*>(dsmem + pad + S * C::STAGE);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * S + 1);
  const uint32_t tiles_u = raw + pad;
  const uint32_t full_u = smem_u32(bars), empty_u = full_u + 8 * S, done_u = full_u + 16 * S;

  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full_u + 8 * i) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty_u + 8 * i) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done_u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(C::COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const int m0 = blockIdx.y * tc::BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * g.kchunk, kend = min(g.K, kbeg + g.kchunk);
  const int nk = kend > kbeg ? (kend - kbeg + tc::BK - 1) / tc::BK : 0;
  int bad = 0;  // this thread's bounded wait ran out

  if (warp == 0 && lane == 0) {
    // ---------------- producer
    int kt = 0;
    for (; kt < nk; ++kt) {
      const int st = kt % S;
      // slot st was last read by the MMAs of step kt - S
      if (kt >= S && !mbar_wait(empty_u + 8 * st, ((kt / S) - 1) & 1)) {
        bad = 1;
        break;
      }
      const uint32_t bar = full_u + 8 * st;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                   "r"(C::STAGE)
                   : "memory");
      const uint32_t sa = tiles_u + st * C::STAGE, sb = sa + C::A_TILE;
      const int k0 = kbeg + kt * tc::BK;  // a multiple of 64 elements (128 B)
      tma_2d(sa, &tmA, k0, m0, bar);
      tma_2d(sb, &tmB, k0, n0, bar);
    }
    if (bad) {
      // let the copies already requested land before the CTA's memory goes away
      for (int k2 = kt - 1; k2 >= 0 && k2 >= kt - S; --k2)
        mbar_wait(full_u + 8 * (k2 % S), (k2 / S) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    for (int kt = 0; kt < nk; ++kt) {
      const int st = kt % S;
      if (!mbar_wait(full_u + 8 * st, (kt / S) & 1)) {
        bad = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = tiles_u + st * C::STAGE, b0 = a0 + C::A_TILE;
#pragma unroll
      for (int kk = 0; kk < tc::BK / 16; ++kk) {
        // K = 16 elements = 32 B further along the swizzled 128-B rows
        const uint64_t ad = smem_desc_sw128(a0 + kk * 32, C::SBO);
        const uint64_t bd = smem_desc_sw128(b0 + kk * 32, C::SBO);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(C::IDESC), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              empty_u + 8 * st)
          : "memory");
    }
    // `done` fires once every MMA issued above has completed
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            done_u)
        : "memory");
  }
  __syncwarp();
  // every warp waits for the accumulator (lane 0 polls, the warp follows)
  if (lane == 0 && !bad && !mbar_wait(done_u, 0)) bad = 1;
  const int aborted = __syncthreads_or(bad);
  tc_fence_after();
  if (aborted) {
    if (tid == 0) atomicExch(&g_tc_error, 1);
  } else {
    const int r = m0 + warp * 32 + lane;
    const bool vf = g.Cf && !g.partial && (g.ldc & 3) == 0 && ((uintptr_t)g.Cf & 15) == 0;
    const bool vb = g.Cb && !g.partial && (g.ldcb & 7) == 0 && ((uintptr_t)g.Cb & 15) == 0;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (r >= g.M) continue;
      store_row32(g, r, n0 + c0, blockIdx.z, v, nk > 0, vf, vb);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::COLS)
                 : "memory");
  }
}

// Persistent form (the default): one CTA per SM walks the tiles (z, m, n) with
// stride gridDim.x, in 6 warps with fixed roles, so that the loads and MMAs of
// the next tile overlap the epilogue of the previous one:
//  - warp 0 (one thread): TMA producer over a ring of STAGES slots, as above,
//    the slot/phase counters running on across tiles;
//  - warp 1 (one thread): MMA issuer into one of two accumulators in tensor
//    memory (columns [0, BN) and [BN, 2 BN)), alternating per tile; before
//    reusing one it waits on that accumulator's `tmem_empty` mbarrier, and
//    after a tile's last MMA it commits to its `tmem_full`;
//  - warps 2-5 (the epilogue): wait on `tmem_full`, read their lane quarter
//    (warp w reads lanes 32 (w mod 4) .. +31) with tcgen05.ld, store, and free
//    the accumulator (one arrival on `tmem_empty` after a named barrier).
// Every wait is bounded and also ends when another role has given up (a
// shared flag); the CTA then records the error, lets its copies in flight land
// (bounded), frees its tensor memory and returns.
namespace tcp {
constexpr int THREADS = 192;
// band mode: 130 rows of 128 B (64 channels) per band, each band in its own
// 1024-byte aligned slot (the 128-byte swizzle repeats every 8 rows)
constexpr int BAND_ROWS = 130;
constexpr int BAND_BYTES = BAND_ROWS * 128;
constexpr int BAND_SLOT = 17 * 1024;
constexpr int SMEM_MAX = 226 * 1024;  // dynamic; the 227 KB per-block limit includes static
template <int BN>
struct Cfg {
  using T = tc::Cfg<BN>;
  static constexpr int STAGE = T::STAGE;
  // one CTA per SM: a ring of about 200 KB (10, 8, 6 slots for BN = 32, 64,
  // 128) keeps enough loads in flight to cover the L2 latency of narrow tiles
  static constexpr int STAGES = (200 * 1024) / STAGE;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 512;
  static constexpr uint32_t COLS = 2 * BN < 32 ? 32 : 2 * BN;  // two accumulators
};
}  // namespace tcp

// bounded wait that also gives up once *abort is set
__device__ __forceinline__ bool mbar_wait_ab(uint32_t bar, uint32_t parity,
                                             const volatile int* abort) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t deadline = globaltimer_ns() + 1000000000ull;
  for (uint32_t it = 0; it < (1u << 24); ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 255 && (*abort || globaltimer_ns() > deadline)) return false;
  }
  return false;
}

template <int BN, bool BAND = false>
__global__ void __launch_bounds__(tcp::THREADS, 1) k_gemm_tcp(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmArgs g,
    int tiles_m, int tiles_n, int tiles_z) {
  using C = tcp::Cfg<BN>;
  using T = tc::Cfg<BN>;
  // ring slots with a full/empty mbarrier pair: the STAGES (A + B) slots, or in
  // band mode AG band groups (pairs 0 .. AG - 1) followed by BS B slots, or by
  // one pair for the resident weights (BS = 0: all 9 C / 64 B tiles loaded once)
  const int cpt = BAND ? g.conv_c >> 6 : 0;  // 64-channel chunks (band mode)
  const int AG = BAND ? g.conv_ag : 1;  // (1, 1: unused outside band mode)
  const int BS = BAND ? g.conv_bs : 1;
  const bool bres = BAND && BS == 0;
  const int S = BAND ? AG + (bres ? 1 : BS) : C::STAGES;
  const uint32_t group_bytes = (uint32_t)cpt * tcp::BAND_SLOT;
  const uint32_t bring_bytes = bres ? 9u * cpt * T::B_TILE : (uint32_t)BS * T::B_TILE;
  const uint32_t ring_bytes = BAND ? AG * group_bytes + bring_bytes
                                   : (uint32_t)(C::STAGES * C::STAGE);
  extern __shared__ uint8_t dsmem[];
  __shared__ int s_abort;
  __shared__ int s_issued, s_consumed;  // k-steps requested by the producer / read by the MMAs
  __shared__ int s_issued_b, s_consumed_b;  // band mode: B loads (the above count band groups)
  __shared__ int s_ep_ok[4];            // per epilogue warp: its accumulator wait succeeded
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t raw = smem_u32(dsmem);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint64_t* bars = reinterpret_cast<uint64_t*>(dsmem + pad + ring_bytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * S + 5);
  const uint32_t tiles_u = raw + pad;
  const uint32_t bring_u = tiles_u + AG * group_bytes;  // band mode: the B ring or resident B
  const uint32_t full_u = smem_u32(bars), empty_u = full_u + 8 * S;
  const uint32_t tfull_u = full_u + 16 * S, tempty_u = tfull_u + 16;  // two of each
  const uint32_t mdone_u = tempty_u + 16;  // the MMA thread's last commit
  const volatile int* abort = &s_abort;

  if (tid == 0) {
    s_abort = 0;
    s_issued = 0;
    s_consumed = 0;
    s_issued_b = 0;
    s_consumed_b = 0;
    for (int i = 0; i < S; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full_u + 8 * i) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty_u + 8 * i) : "memory");
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tfull_u + 8 * i) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tempty_u + 8 * i) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mdone_u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(C::COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int ntiles = tiles_m * tiles_n * tiles_z;
  // tile t -> (z, m, n), n fastest: neighbouring CTAs share the A tile in L2
  auto coords = [&](int t, int& m0, int& n0, int& kbeg, int& nk) {
    const int n = t % tiles_n, m = (t / tiles_n) % tiles_m, z = t / (tiles_n * tiles_m);
    m0 = m * tc::BM;
    n0 = n * BN;
    kbeg = z * g.kchunk;
    const int kend = min(g.K, kbeg + g.kchunk);
    nk = kend > kbeg ? (kend - kbeg + tc::BK - 1) / tc::BK : 0;
    return z;
  };

  if (warp == 0) {
    if (lane == 0 && BAND) {
      // ---------------- producer, band mode: per tile and input row dy, one
      // band of 130 pixels per 64-channel chunk (a group); the weights of the
      // three taps (dy, dx) of every chunk follow in the im2col K order, or
      // (resident weights) all 9 C / 64 weight tiles are loaded once up front
      int ga = 0, gb = 0;  // band groups / B loads issued so far (all tiles)
      bool ok = true;
      if (bres) {
        const uint32_t bbar = full_u + 8 * AG;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bbar),
                     "r"(bring_bytes)
                     : "memory");
        for (int j = 0; j < 9 * cpt; ++j) tma_2d(bring_u + j * T::B_TILE, &tmB, j << 6, 0, bbar);
        gb = 1;
      }
      for (int t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x) {
        int m0, n0, kbeg, nk;
        coords(t, m0, n0, kbeg, nk);
        const int hw = g.conv_h * g.conv_w, b0 = m0 / hw, rem = m0 - b0 * hw;
        const int h0 = rem / g.conv_w, w0 = rem - h0 * g.conv_w;
        for (int dy = 0; dy < 3 && ok; ++dy, ++ga) {
          const int as = ga % AG;
          if (ga >= AG && !mbar_wait_ab(empty_u + 8 * as, ((ga / AG) - 1) & 1, abort)) {
            ok = false;
            break;
          }
          const uint32_t abar = full_u + 8 * as;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(abar),
                       "r"(cpt * tcp::BAND_BYTES)
                       : "memory");
          for (int c = 0; c < cpt; ++c)
            tma_4d(tiles_u + as * group_bytes + c * tcp::BAND_SLOT, &tmA, c << 6, w0 - 1,
                   h0 + dy - 1, b0, abar);
          if (bres) continue;
          for (int dx = 0; dx < 3 && ok; ++dx)
            for (int c = 0; c < cpt; ++c, ++gb) {
              const int bs = gb % BS;
              if (gb >= BS &&
                  !mbar_wait_ab(empty_u + 8 * (AG + bs), ((gb / BS) - 1) & 1, abort)) {
                ok = false;
                break;
              }
              const uint32_t bbar = full_u + 8 * (AG + bs);
              asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bbar),
                           "r"(T::B_TILE)
                           : "memory");
              tma_2d(bring_u + bs * T::B_TILE, &tmB, ((dy * 3 + dx) * cpt + c) << 6, n0, bbar);
            }
        }
      }
      if (!ok) s_abort = 1;
      s_issued = ga;
      s_issued_b = gb;
    } else if (lane == 0) {
      // ---------------- producer
      int gk = 0;  // k-steps issued so far (all tiles)
      for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
        int m0, n0, kbeg, nk;
        coords(t, m0, n0, kbeg, nk);
        for (int kt = 0; kt < nk; ++kt, ++gk) {
          const int st = gk % S;
          if (gk >= S && !mbar_wait_ab(empty_u + 8 * st, ((gk / S) - 1) & 1, abort)) {
            s_abort = 1;
            break;
          }
          const uint32_t bar = full_u + 8 * st;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                       "r"(C::STAGE)
                       : "memory");
          const uint32_t sa = tiles_u + st * C::STAGE;
          const int k0 = kbeg + kt * tc::BK;  // a multiple of 64 elements (128 B)
          if (g.conv_c) {
            // implicit convolution: the tap's shifted box of 128 pixels
            const int cpt = g.conv_c >> 6, tap = kt / cpt, c0 = (kt - tap * cpt) << 6;
            const int hw = g.conv_h * g.conv_w, b0 = m0 / hw, rem = m0 - b0 * hw;
            const int h0 = rem / g.conv_w, w0 = rem - h0 * g.conv_w;
            tma_4d(sa, &tmA, c0, w0 + tap % 3 - 1, h0 + tap / 3 - 1, b0, bar);
          } else {
            tma_2d(sa, &tmA, k0, m0, bar);
          }
          tma_2d(sa + T::A_TILE, &tmB, k0, n0, bar);
        }
      }
      s_issued = gk;
    }
  } else if (warp == 1) {
    if (lane == 0 && BAND) {
      // ---------------- MMA issuer, band mode: tap (dy, dx) of chunk c reads
      // rows dx .. dx + 127 of band (dy, c), i.e. the descriptor starts dx rows
      // (128 B each) into the band; the swizzle follows the absolute address
      int ga = 0, gb = 0, it = 0;
      bool ok = true;
      if (bres) {
        if (!mbar_wait_ab(full_u + 8 * AG, 0, abort)) ok = false;
        else gb = 1;
      }
      for (int t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x, ++it) {
        const int acc = it & 1;
        if (it >= 2 && !mbar_wait_ab(tempty_u + 8 * acc, ((it >> 1) - 1) & 1, abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * BN);
        uint32_t accum = 0u;
        for (int dy = 0; dy < 3 && ok; ++dy, ++ga) {
          const int as = ga % AG;
          if (!mbar_wait_ab(full_u + 8 * as, (ga / AG) & 1, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t abase = tiles_u + as * group_bytes;
          for (int dx = 0; dx < 3 && ok; ++dx)
            for (int c = 0; c < cpt; ++c) {
              const int bs = bres ? 0 : gb % BS;
              if (!bres) {
                if (!mbar_wait_ab(full_u + 8 * (AG + bs), (gb / BS) & 1, abort)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
              }
              const uint32_t a0 = abase + c * tcp::BAND_SLOT + dx * 128;
              const uint32_t b0 = bres ? bring_u + ((dy * 3 + dx) * cpt + c) * T::B_TILE
                                       : bring_u + bs * T::B_TILE;
#pragma unroll
              for (int kk = 0; kk < tc::BK / 16; ++kk) {
                const uint64_t ad = smem_desc_sw128(a0 + kk * 32, T::SBO);
                const uint64_t bd = smem_desc_sw128(b0 + kk * 32, T::SBO);
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                    "l"(ad), "l"(bd), "r"(T::IDESC), "r"(accum)
                    : "memory");
                accum = 1u;
              }
              if (!bres) {
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        empty_u + 8 * (AG + bs))
                    : "memory");
                ++gb;
              }
            }
          // the band group is free once these MMAs have read it
          if (ok)
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    empty_u + 8 * as)
                : "memory");
        }
        if (!ok) break;
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                tfull_u + 8 * acc)
            : "memory");
      }
      if (!ok) s_abort = 1;
      s_consumed = ga;
      s_consumed_b = gb;
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              mdone_u)
          : "memory");
      if (!mbar_wait(mdone_u, 0)) s_abort = 1;
    } else if (lane == 0) {
      // ---------------- MMA issuer
      int gk = 0, it = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x, ++it) {
        int m0, n0, kbeg, nk;
        coords(t, m0, n0, kbeg, nk);
        const int acc = it & 1;
        // the epilogue of tile it - 2 has read this accumulator
        if (it >= 2 && !mbar_wait_ab(tempty_u + 8 * acc, ((it >> 1) - 1) & 1, abort)) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * BN);
        bool ok = true;
        for (int kt = 0; kt < nk; ++kt, ++gk) {
          const int st = gk % S;
          if (!mbar_wait_ab(full_u + 8 * st, (gk / S) & 1, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = tiles_u + st * C::STAGE, b0 = a0 + T::A_TILE;
#pragma unroll
          for (int kk = 0; kk < tc::BK / 16; ++kk) {
            const uint64_t ad = smem_desc_sw128(a0 + kk * 32, T::SBO);
            const uint64_t bd = smem_desc_sw128(b0 + kk * 32, T::SBO);
            const uint32_t accum = (kt > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                "l"(ad), "l"(bd), "r"(T::IDESC), "r"(accum)
                : "memory");
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  empty_u + 8 * st)
              : "memory");
        }
        if (!ok) {
          s_abort = 1;
          break;
        }
        // the accumulator is complete once these MMAs are
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                tfull_u + 8 * acc)
            : "memory");
      }
      s_consumed = gk;
      // every MMA this thread issued has completed before the CTA moves on
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              mdone_u)
          : "memory");
      if (!mbar_wait(mdone_u, 0)) s_abort = 1;
    }
  } else {
    // ---------------- epilogue, warps 2-5: lane quarter q = warp mod 4
    const int q = warp & 3;
    const bool vf = g.Cf && !g.partial && (g.ldc & 3) == 0 && ((uintptr_t)g.Cf & 15) == 0;
    const bool vb = g.Cb && !g.partial && (g.ldcb & 7) == 0 && ((uintptr_t)g.Cb & 15) == 0;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      int m0, n0, kbeg, nk;
      const int z = coords(t, m0, n0, kbeg, nk);
      const int acc = it & 1;
      int ready = 1;
      if (lane == 0) ready = mbar_wait_ab(tfull_u + 8 * acc, (it >> 1) & 1, abort) ? 1 : 0;
      ready = __shfl_sync(0xffffffffu, ready, 0);
      // the four epilogue warps decide together (no warp leaves the named barrier alone)
      if (lane == 0) s_ep_ok[q] = ready;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      const int all_ok = s_ep_ok[0] & s_ep_ok[1] & s_ep_ok[2] & s_ep_ok[3];
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (!all_ok) {
        if (warp == 2 && lane == 0) s_abort = 1;
        break;
      }
      tc_fence_after();
      const int r = m0 + q * 32 + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c0), v);
        if (r < g.M) store_row32(g, r, n0 + c0, z, v, nk > 0, vf, vb);
      }
      // all four epilogue warps are done with this accumulator
      tc_fence_before();
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (warp == 2 && lane == 0)
        asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(tempty_u + 8 * acc)
                     : "memory");
    }
  }
  __syncwarp();
  __syncthreads();
  if (s_abort) {
    if (tid == 0) {
      atomicExch(&g_tc_error, 1);
      // let the copies still in flight land before the CTA's memory goes away
      if (BAND) {
        for (int k2 = s_consumed; k2 < s_issued; ++k2)
          mbar_wait(full_u + 8 * (k2 % AG), (k2 / AG) & 1);
        if (bres) {
          if (s_issued_b > s_consumed_b) mbar_wait(full_u + 8 * AG, 0);
        } else {
          for (int k2 = s_consumed_b; k2 < s_issued_b; ++k2)
            mbar_wait(full_u + 8 * (AG + k2 % BS), (k2 / BS) & 1);
        }
      } else {
        for (int k2 = s_consumed; k2 < s_issued; ++k2)
          mbar_wait(full_u + 8 * (k2 % S), (k2 / S) & 1);
      }
    }
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::COLS)
                 : "memory");
  }
}

// split-K: C = sum over slices z (fixed order) of partial[z]; then bias, act
__global__ void k_splitk_reduce(const float* __restrict__ partial, int splits, int M, int N,
                                float* __restrict__ Cf, int ldc, const float* __restrict__ bias,
                                int act, int accumulate) {
  const int64_t total = (int64_t)M * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int z = 0; z < splits; ++z) v += partial[(int64_t)z * total + i];
    const int r = (int)(i / N), c = (int)(i % N);
    if (bias) v += bias[c];
    v = act_fwd(v, act);
    float* p = Cf + (size_t)r * ldc + c;
    *p = accumulate ? *p + v : v;
  }
}

// ------------------------------------------------------------------ conv helpers
// im2col: col[p][(kh*3 + kw)*C + c] = X[b][h + kh - 1][w + kw - 1][c] (zero outside)
__global__ void k_im2col(const bf16* __restrict__ X, int B, int H, int W, int C, int cs,
                         bf16* __restrict__ col) {
  const int64_t total = (int64_t)B * H * W * 9 * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t r = i / C;
    const int tap = (int)(r % 9);
    const int64_t p = r / 9;
    const int w = (int)(p % W), h = (int)((p / W) % H), b = (int)(p / ((int64_t)W * H));
    const int hh = h + tap / 3 - 1, ww = w + tap % 3 - 1;
    bf16 v = __float2bfloat16_rn(0.f);
    if (hh >= 0 && hh < H && ww >= 0 && ww < W) v = X[(((int64_t)b * H + hh) * W + ww) * cs + c];
    col[i] = v;
  }
}

// transposed im2col: colT[(kh*3 + kw)*C + c][p] (pixels contiguous)
__global__ void k_im2col_t(const bf16* __restrict__ X, int B, int H, int W, int C, int cs,
                           bf16* __restrict__ colT) {
  const int64_t P = (int64_t)B * H * W, total = P * 9 * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i % P;
    const int64_t k = i / P;
    const int c = (int)(k % C), tap = (int)(k / C);
    const int w = (int)(p % W), h = (int)((p / W) % H), b = (int)(p / ((int64_t)W * H));
    const int hh = h + tap / 3 - 1, ww = w + tap % 3 - 1;
    bf16 v = __float2bfloat16_rn(0.f);
    if (hh >= 0 && hh < H && ww >= 0 && ww < W) v = X[(((int64_t)b * H + hh) * W + ww) * cs + c];
    colT[i] = v;
  }
}

// Vector forms (16-byte chunks of 8 channels; used when C, cs are multiples of
// 8 and the buffers 16-byte aligned): one thread per (pixel, tap, chunk).
__global__ void k_im2col_v8(const bf16* __restrict__ X, int B, int H, int W, int C8, int cs,
                            bf16* __restrict__ col) {
  const int64_t total = (int64_t)B * H * W * 9 * C8;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c8 = (int)(i % C8);
    const int64_t r = i / C8;
    const int tap = (int)(r % 9);
    const int64_t p = r / 9;
    const int w = (int)(p % W);
    const int64_t t = p / W;
    const int h = (int)(t % H), b = (int)(t / H);
    const int hh = h + tap / 3 - 1, ww = w + tap % 3 - 1;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (hh >= 0 && hh < H && ww >= 0 && ww < W)
      v = *reinterpret_cast<const uint4*>(X + (((int64_t)b * H + hh) * W + ww) * cs + c8 * 8);
    *reinterpret_cast<uint4*>(col + i * 8) = v;
  }
}

// transposed: thread (row group k8 = tap*C8 + c8, pixel p), pixels fastest, so
// each of the 8 rows it writes is written coalesced across the warp
__global__ void k_im2col_t_v8(const bf16* __restrict__ X, int B, int H, int W, int C8, int cs,
                              bf16* __restrict__ colT) {
  const int64_t P = (int64_t)B * H * W, total = P * 9 * C8;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i % P;
    const int k8 = (int)(i / P);
    const int c8 = k8 % C8, tap = k8 / C8;
    const int w = (int)(p % W);
    const int64_t t = p / W;
    const int h = (int)(t % H), b = (int)(t / H);
    const int hh = h + tap / 3 - 1, ww = w + tap % 3 - 1;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (hh >= 0 && hh < H && ww >= 0 && ww < W)
      v = *reinterpret_cast<const uint4*>(X + (((int64_t)b * H + hh) * W + ww) * cs + c8 * 8);
    const bf16* e = reinterpret_cast<const bf16*>(&v);
    bf16* dst = colT + ((int64_t)tap * C8 * 8 + c8 * 8) * P + p;
#pragma unroll
    for (int j = 0; j < 8; ++j) dst[j * P] = e[j];
  }
}

// col2im with 4 channels per thread (C, cs multiples of 4, 16-byte aligned)
__global__ void k_col2im_v4(const float* __restrict__ dcol, int B, int H, int W, int C4,
                            float* __restrict__ dX, int cs) {
  const int64_t total = (int64_t)B * H * W * C4;
  const int C = C4 * 4;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c4 = (int)(i % C4);
    const int64_t p = i / C4;
    const int w = (int)(p % W);
    const int64_t t = p / W;
    const int h = (int)(t % H), b = (int)(t / H);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int ho = h - (tap / 3 - 1), wo = w - (tap % 3 - 1);  // output pixel reading (h, w)
      if (ho >= 0 && ho < H && wo >= 0 && wo < W) {
        const float4 q = *reinterpret_cast<const float4*>(
            dcol + ((((int64_t)b * H + ho) * W + wo) * 9 + tap) * C + c4 * 4);
        s.x += q.x; s.y += q.y; s.z += q.z; s.w += q.w;
      }
    }
    *reinterpret_cast<float4*>(dX + p * cs + c4 * 4) = s;
  }
}

// col2im: dX[b][h][w][c] = sum over taps of dcol[pixel that reads (h, w)][tap][c]
__global__ void k_col2im(const float* __restrict__ dcol, int B, int H, int W, int C,
                         float* __restrict__ dX, int cs) {
  const int64_t total = (int64_t)B * H * W * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t p = i / C;
    const int w = (int)(p % W), h = (int)((p / W) % H), b = (int)(p / ((int64_t)W * H));
    float s = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int ho = h - (tap / 3 - 1), wo = w - (tap % 3 - 1);  // output pixel reading (h, w)
      if (ho >= 0 && ho < H && wo >= 0 && wo < W)
        s += dcol[((((int64_t)b * H + ho) * W + wo) * 9 + tap) * C + c];
    }
    dX[p * cs + c] = s;
  }
}

// dst[n][m] = src[m][n] (BF16, src row stride lds)
// Wf[ci][tap][co] = Wt[co][8 - tap][ci]: the weights of the adjoint of a 3x3
// convolution (dX = conv3x3(dY, Wf) with the taps mirrored and the channel
// roles swapped)
__global__ void k_conv_flip(const bf16* __restrict__ Wt, int Co, int Ci, bf16* __restrict__ Wf) {
  const int64_t n = (int64_t)Co * 9 * Ci;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int ci = (int)(i % Ci), tap = (int)((i / Ci) % 9), co = (int)(i / (9 * (int64_t)Ci));
    Wf[((int64_t)ci * 9 + (8 - tap)) * Co + co] = Wt[i];
  }
}

__global__ void k_transpose(const bf16* __restrict__ src, int M, int N, int lds,
                            bf16* __restrict__ dst) {
  __shared__ bf16 t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int m = by + j, n = bx + threadIdx.x;
    if (m < M && n < N) t[j][threadIdx.x] = src[(size_t)m * lds + n];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int n = bx + j, m = by + threadIdx.x;
    if (m < M && n < N) dst[(size_t)n * M + m] = t[threadIdx.x][j];
  }
}

// 2x2 average pool (fwd) / its adjoint (bwd), nearest 2x upsample (fwd) / adjoint (bwd)
__global__ void k_pool(const bf16* __restrict__ X, int B, int H, int W, int C, int csx,
                       bf16* __restrict__ Y, int csy) {
  const int Ho = H / 2, Wo = W / 2;
  const int64_t total = (int64_t)B * Ho * Wo * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t p = i / C;
    const int w = (int)(p % Wo), h = (int)((p / Wo) % Ho), b = (int)(p / ((int64_t)Wo * Ho));
    float s = 0.f;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx)
        s += __bfloat162float(X[(((int64_t)b * H + 2 * h + dy) * W + 2 * w + dx) * csx + c]);
    Y[p * csy + c] = __float2bfloat16_rn(0.25f * s);
  }
}

__global__ void k_pool_bwd(const float* __restrict__ dY, int B, int H, int W, int C, int csy,
                           float* __restrict__ dX, int csx, int accumulate) {
  const int64_t total = (int64_t)B * H * W * C;  // H, W of the input (fine) grid
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t p = i / C;
    const int w = (int)(p % W), h = (int)((p / W) % H), b = (int)(p / ((int64_t)W * H));
    const float v = 0.25f * dY[(((int64_t)b * (H / 2) + h / 2) * (W / 2) + w / 2) * csy + c];
    float* d = dX + p * csx + c;
    *d = accumulate ? *d + v : v;
  }
}

__global__ void k_upsample(const bf16* __restrict__ X, int B, int H, int W, int C, int csx,
                           bf16* __restrict__ Y, int csy) {
  const int64_t total = (int64_t)B * 2 * H * 2 * W * C;  // output grid 2H x 2W
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t p = i / C;
    const int w = (int)(p % (2 * W)), h = (int)((p / (2 * W)) % (2 * H));
    const int b = (int)(p / ((int64_t)4 * W * H));
    Y[p * csy + c] = X[(((int64_t)b * H + h / 2) * W + w / 2) * csx + c];
  }
}

__global__ void k_upsample_bwd(const float* __restrict__ dY, int B, int H, int W, int C, int csy,
                               float* __restrict__ dX, int csx) {
  const int64_t total = (int64_t)B * H * W * C;  // coarse grid
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t p = i / C;
    const int w = (int)(p % W), h = (int)((p / W) % H), b = (int)(p / ((int64_t)W * H));
    float s = 0.f;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx)
        s += dY[(((int64_t)b * 2 * H + 2 * h + dy) * 2 * W + 2 * w + dx) * csy + c];
    dX[p * csx + c] = s;
  }
}

// gradient through the activation: g *= f'(z), with f' read from the output y
// (leaky ReLU: 1 where y > 0, else the slope); writes FP32 and a BF16 copy
__global__ void k_act_bwd(float* __restrict__ g, const bf16* __restrict__ y, int64_t rows, int C,
                          int csg, int csy, int act, bf16* __restrict__ gb, int csb) {
  const int64_t total = rows * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t r = i / C;
    float v = g[r * csg + c];
    if (act == 1 && !(__bfloat162float(y[r * csy + c]) > 0.f)) v *= 0.02f;
    g[r * csg + c] = v;
    if (gb) gb[r * csb + c] = __float2bfloat16_rn(v);
  }
}

// db[c] = sum over rows of g[r][c] (fixed order per channel)
// Two-pass column sums for wide row counts: pass 1, block (channel group of 32,
// row chunk) with 8 warps striding the chunk's rows (coalesced 128-byte row
// segments), partial sums to a fixed scratch; pass 2 adds the chunks in order
// (deterministic).
constexpr int kBiasChunks = 64, kBiasMaxC = 4096;
__device__ float g_bias_partial[kBiasChunks * kBiasMaxC];

__global__ void __launch_bounds__(256) k_bias_grad_part(const float* __restrict__ g,
                                                        int64_t rows, int C, int cs) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  const int64_t per = (rows + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = blockIdx.y * per, r1 = r0 + per < rows ? r0 + per : rows;
  float s = 0.f;
  if (c < C)
    for (int64_t r = r0 + wp; r < r1; r += 8) s += g[r * cs + c];
  __shared__ float sh[8][32];
  sh[wp][lane] = s;
  __syncthreads();
  if (wp == 0 && c < C) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += sh[k][lane];
    g_bias_partial[(int64_t)blockIdx.y * C + c] = t;
  }
}

__global__ void k_bias_grad_final(int C, int chunks, float* __restrict__ db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  float t = 0.f;
  for (int k = 0; k < chunks; ++k) t += g_bias_partial[(int64_t)k * C + c];
  db[c] = t;
}

__global__ void k_bias_grad(const float* __restrict__ g, int64_t rows, int C, int cs,
                            float* __restrict__ db) {
  const int c = blockIdx.x;
  __shared__ float sh[256];
  float s = 0.f;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) s += g[r * cs + c];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] = sh[0];
}

// loss = mean((pred - target)^2) over rows x C; grad = 2 (pred - target) / count
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ target,
                      int64_t n, float* __restrict__ grad, double* __restrict__ partial) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = pred[i] - target[i];
    s += (double)d * d;
    if (grad) grad[i] = 2.0f * d / (float)n;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_sum(const double* __restrict__ partial, int n, double scale,
                      double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += partial[i];
  *out = s * scale;
}

// Adam on FP32 master weights, refreshes the BF16 copy used by the GEMMs
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, bf16* __restrict__ wb, int64_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2, float wd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i] + wd * w[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void k_cast_bf16(const float* __restrict__ x, int64_t rows, int C, int csx,
                            bf16* __restrict__ y, int csy) {
  const int64_t total = rows * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t r = i / C;
    y[r * csy + c] = __float2bfloat16_rn(x[r * csx + c]);
  }
}

int grid_for(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)(g < 152 * 32 ? (g < 1 ? 1 : g) : 152 * 32);
}

}  // namespace nn
}  // namespace ddflb

using namespace ddflb::nn;

namespace {
ddflb_status launched(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return DDFLB_OK;
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  ddflb::set_error(buf);
  return DDFLB_ECUDA;
}
ddflb_status bad(const char* msg) {
  ddflb::set_error(msg);
  return DDFLB_EINVAL;
}
}  // namespace

namespace {
int g_gemm_path = 0;  // 0: tcgen05 persistent (default), 1: mma.sync, 2: tcgen05 one tile per CTA

// cuTensorMapEncodeTiled from the driver, looked up through the runtime (no
// link-time dependency on the driver library)
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
  }
  return fn;
}

// 2-D map over a row-major BF16 matrix [rows][K] (row stride ld elements):
// boxes of 64 K-elements (128 B) x box_rows rows, 128-byte swizzle, zero fill
// outside
bool make_map(CUtensorMap* m, const void* base, int rows, int K, int ld, int box_rows) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 4-D map over an NHWC BF16 activation [B][H][W][cs] (C channels used): boxes
// of 64 channels x bw x bh x bb pixels, 128-byte swizzle, zero fill outside the
// image (the convolution's padding)
bool make_map_conv(CUtensorMap* m, const void* base, int B, int H, int W, int C, int cs, int bw,
                   int bh, int bb) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)cs * 2, (cuuint64_t)W * cs * 2,
                                 (cuuint64_t)H * W * cs * 2};
  const cuuint32_t box[4] = {64, (cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)bb};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 1;
  }
  return n;
}

template <int BN>
ddflb_status gemm_tcp_bn(const GemmArgs& g, int tm, int tn, int tz, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_gemm_tcp<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tcp::Cfg<BN>::SMEM) != cudaSuccess)
      return launched("gemm tcgen05 attribute");
    attr = true;
  }
  CUtensorMap ma, mb;
  if (!make_map(&ma, g.A, g.M, g.K, g.lda, tc::BM) || !make_map(&mb, g.B, g.N, g.K, g.ldb, BN))
    return bad("gemm: TMA tensor map encoding failed");
  const int ntiles = tm * tn * tz;
  const int grid = ntiles < sm_count() ? ntiles : sm_count();
  k_gemm_tcp<BN><<<grid, tcp::THREADS, tcp::Cfg<BN>::SMEM, s>>>(ma, mb, g, tm, tn, tz);
  return launched("gemm tcgen05 persistent");
}

// 0: bands where W is a multiple of 128 and C >= 128, else per-tap boxes;
// 1: per-tap boxes everywhere
int g_conv_path = 0;

// Implicit 3x3 convolution on the persistent kernel: the A map is 4-D over the
// activation, the B map 2-D over the weights [N][9 C].  Band mode (W a
// multiple of 128): the A map's box is a band of 130 pixels of one row, three
// per tile and 64-channel chunk, each read by the three taps of its row.
template <int BN>
ddflb_status conv_tcp_bn(GemmArgs g, const void* X, int B, int cs, cudaStream_t s) {
  const int tm = g.M / tc::BM, tn = (g.N + BN - 1) / BN;
  const int grid = tm * tn < sm_count() ? tm * tn : sm_count();
  // band mode: the weights stay resident when N fits one tile and they leave
  // room for at least two band groups; else a ring of B slots
  const int cpt = g.conv_c / 64;
  const int group = cpt * tcp::BAND_SLOT, avail = tcp::SMEM_MAX - 1024 - 512;
  const int bres_bytes = 9 * cpt * tc::Cfg<BN>::B_TILE;
  int ag = 0, bs = 0;
  if (tn == 1 && avail - bres_bytes >= 2 * group) {
    ag = (avail - bres_bytes) / group;
  } else {
    bs = 8;
    ag = (avail - bs * tc::Cfg<BN>::B_TILE) / group;
  }
  ag = ag < 6 ? ag : 6;
  // measured on the U-Net's layers: bands pay only with two or more channel
  // chunks (128 x 128 x 128 -> 64: -9 %); with one chunk their shifted operand
  // reads cost more than the loads they save, and the per-tap boxes are faster
  if (g_conv_path == 0 && cpt >= 2 && g.conv_bw == 128 && g.conv_bh == 1 && g.conv_bb == 1 &&
      ag >= 2) {
    static bool battr = false;
    if (!battr) {
      if (cudaFuncSetAttribute(k_gemm_tcp<BN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               tcp::SMEM_MAX) != cudaSuccess)
        return launched("conv tcgen05 band attribute");
      battr = true;
    }
    CUtensorMap ma, mb;
    g.conv_ag = ag;
    g.conv_bs = bs;
    if (make_map_conv(&ma, X, B, g.conv_h, g.conv_w, g.conv_c, cs, tcp::BAND_ROWS, 1, 1) &&
        make_map(&mb, g.B, g.N, g.K, g.ldb, BN)) {
      const int smem = ag * group + (bs ? bs * tc::Cfg<BN>::B_TILE : bres_bytes) + 1024 + 512;
      k_gemm_tcp<BN, true><<<grid, tcp::THREADS, smem, s>>>(ma, mb, g, tm, tn, 1);
      return launched("conv3x3 tcgen05 bands");
    }
    // a band map the driver does not encode: per-tap boxes below
  }
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_gemm_tcp<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tcp::Cfg<BN>::SMEM) != cudaSuccess)
      return launched("conv tcgen05 attribute");
    attr = true;
  }
  g.conv_ag = 0;
  g.conv_bs = 0;
  CUtensorMap ma, mb;
  if (!make_map_conv(&ma, X, B, g.conv_h, g.conv_w, g.conv_c, cs, g.conv_bw, g.conv_bh,
                     g.conv_bb) ||
      !make_map(&mb, g.B, g.N, g.K, g.ldb, BN))
    return bad("conv3x3: TMA tensor map encoding failed");
  k_gemm_tcp<BN><<<grid, tcp::THREADS, tcp::Cfg<BN>::SMEM, s>>>(ma, mb, g, tm, tn, 1);
  return launched("conv3x3 tcgen05");
}

template <int BN>
ddflb_status gemm_tc_bn(const GemmArgs& g, dim3 grid, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_gemm_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc::Cfg<BN>::SMEM) != cudaSuccess)
      return launched("gemm tcgen05 attribute");
    attr = true;
  }
  CUtensorMap ma, mb;
  if (!make_map(&ma, g.A, g.M, g.K, g.lda, tc::BM) || !make_map(&mb, g.B, g.N, g.K, g.ldb, BN))
    return bad("gemm: TMA tensor map encoding failed");
  k_gemm_tc<BN><<<grid, tc::THREADS, tc::Cfg<BN>::SMEM, s>>>(ma, mb, g);
  return launched("gemm tcgen05");
}

// N tile: the smallest of 32, 64, 128 that covers N (wider N: 128-column tiles)
ddflb_status gemm_tc(GemmArgs g, int splits, bool persistent, cudaStream_t s) {
  int kchunk = g.K;
  if (splits > 1) {
    kchunk = (g.K + splits - 1) / splits;
    kchunk = (kchunk + tc::BK - 1) / tc::BK * tc::BK;
  }
  const int z = (g.K + kchunk - 1) / kchunk;
  g.kchunk = kchunk;
  const int bn = g.N <= 32 ? 32 : g.N <= 64 ? 64 : 128;
  dim3 grid((g.N + bn - 1) / bn, (g.M + tc::BM - 1) / tc::BM, z);
  ddflb_status st;
  // with no more tiles than SMs every CTA would own one tile anyway: the
  // one-tile kernel has the lighter set-up
  if (persistent && (int64_t)grid.x * grid.y * grid.z > sm_count())
    st = bn == 32   ? gemm_tcp_bn<32>(g, grid.y, grid.x, z, s)
         : bn == 64 ? gemm_tcp_bn<64>(g, grid.y, grid.x, z, s)
                    : gemm_tcp_bn<128>(g, grid.y, grid.x, z, s);
  else
    st = bn == 32   ? gemm_tc_bn<32>(g, grid, s)
         : bn == 64 ? gemm_tc_bn<64>(g, grid, s)
                    : gemm_tc_bn<128>(g, grid, s);
  if (st != DDFLB_OK || splits == 1) return st;
  k_splitk_reduce<<<grid_for((int64_t)g.M * g.N), 256, 0, s>>>(g.partial, z, g.M, g.N, g.Cf, g.ldc,
                                                               g.bias, g.act, g.accumulate);
  return launched("gemm tcgen05 split-K");
}
}  // namespace

extern "C" {

ddflb_status ddflb_nn_set_gemm_path(int32_t path) {
  if (path < 0 || path > 2)
    return bad("gemm path must be 0 (tcgen05 persistent), 1 (mma.sync) or 2 (tcgen05, one tile per CTA)");
  g_gemm_path = path;
  return DDFLB_OK;
}

ddflb_status ddflb_nn_take_error(int32_t* error, void* stream) {
  if (!error) return bad("take_error: NULL output");
  int* dev = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&dev, g_tc_error);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(error, dev, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev, 0, sizeof(int), (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) {
    ddflb::set_error(cudaGetErrorString(e));
    return DDFLB_ECUDA;
  }
  return DDFLB_OK;
}

ddflb_status ddflb_nn_gemm(const void* A, const void* B, int32_t M, int32_t N, int32_t K,
                           int32_t lda, int32_t ldb, float* Cf, int32_t ldc, void* Cb,
                           int32_t ldcb, const float* bias, int32_t act, int32_t accumulate,
                           int32_t splits, float* partial, void* stream) {
  if (!A || !B || M <= 0 || N <= 0 || K <= 0 || (!Cf && !Cb)) return bad("gemm: bad arguments");
  if (K % 8 || lda % 8 || ldb % 8 || ((uintptr_t)A % 16) || ((uintptr_t)B % 16))
    return bad("gemm: K, lda, ldb must be multiples of 8 and A, B 16-byte aligned");
  if (lda < K || ldb < K || (Cf && ldc < N) || (Cb && ldcb < N)) return bad("gemm: leading dims");
  if (act < 0 || act > 1) return bad("gemm: act must be 0 (none) or 1 (leaky ReLU)");
  if (splits < 1) return bad("gemm: splits < 1");
  cudaStream_t s = (cudaStream_t)stream;
  if (splits > 1 && (!Cf || Cb || !partial))
    return bad("gemm: split-K needs Cf and partial (and no Cb)");
  if (g_gemm_path == 0 || g_gemm_path == 2) {
    GemmArgs g{(const bf16*)A, (const bf16*)B, M, N, K, lda, ldb, splits > 1 ? nullptr : Cf,
               splits > 1 ? nullptr : (bf16*)Cb, ldc, ldcb, bias, act, accumulate, K,
               splits > 1 ? partial : nullptr};
    if (splits > 1) g.Cf = Cf;  // read by the split-K reduction only
    return gemm_tc(g, splits, g_gemm_path == 0, s);
  }
  if (splits == 1) {
    GemmArgs g{(const bf16*)A, (const bf16*)B, M, N, K, lda, ldb, Cf, (bf16*)Cb, ldc, ldcb,
               bias, act, accumulate, K, nullptr};
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm<<<grid, 256, 0, s>>>(g);
    return launched("gemm");
  }
  if (!Cf || Cb || !partial) return bad("gemm: split-K needs Cf and partial (and no Cb)");
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  const int z = (K + kchunk - 1) / kchunk;  // <= splits slices of the partial buffer
  GemmArgs g{(const bf16*)A, (const bf16*)B, M, N, K, lda, ldb, nullptr, nullptr, 0, 0, nullptr,
             0, 0, kchunk, partial};
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, z);
  k_gemm<<<grid, 256, 0, s>>>(g);
  k_splitk_reduce<<<grid_for((int64_t)M * N), 256, 0, s>>>(partial, z, M, N, Cf, ldc, bias, act,
                                                           accumulate);
  return launched("gemm split-K");
}

ddflb_status ddflb_nn_conv3x3(const void* X, int32_t B, int32_t H, int32_t W, int32_t C,
                              int32_t cs, const void* Wt, int32_t N, float* Cf, int32_t ldc,
                              void* Cb, int32_t ldcb, const float* bias, int32_t act,
                              int32_t accumulate, void* stream) {
  if (!X || !Wt || B <= 0 || H <= 0 || W <= 0 || N <= 0 || (!Cf && !Cb))
    return bad("conv3x3: bad arguments");
  if (C % 64 || cs < C || cs % 8 || ((uintptr_t)X % 16) || ((uintptr_t)Wt % 16))
    return bad("conv3x3: C must be a multiple of 64, cs a multiple of 8 (>= C), X and Wt "
               "16-byte aligned");
  if ((Cf && ldc < N) || (Cb && ldcb < N)) return bad("conv3x3: leading dims");
  if (act < 0 || act > 1) return bad("conv3x3: act must be 0 (none) or 1 (leaky ReLU)");
  // a tile of 128 consecutive pixels must be one box (w, h, image)
  const int bw = W < 128 ? W : 128;
  const int bh = 128 / bw < H ? 128 / bw : H;
  const int bb = 128 / (bw * bh);
  if (128 % bw || (W >= 128 && W % 128) || H % bh || bw * bh * bb != 128 || B % bb ||
      ((int64_t)B * H * W) % 128 || (int64_t)B * H * W > INT32_MAX)
    return bad("conv3x3: 128-pixel tiles need W a divisor of 128 or a multiple of it, and whole "
               "boxes of rows and images");
  GemmArgs g{};
  g.A = (const bf16*)X;
  g.B = (const bf16*)Wt;
  g.M = B * H * W;
  g.N = N;
  g.K = 9 * C;
  g.lda = 9 * C;
  g.ldb = 9 * C;
  g.Cf = Cf;
  g.Cb = (bf16*)Cb;
  g.ldc = ldc;
  g.ldcb = ldcb;
  g.bias = bias;
  g.act = act;
  g.accumulate = accumulate;
  g.kchunk = g.K;
  g.partial = nullptr;
  g.conv_c = C;
  g.conv_w = W;
  g.conv_h = H;
  g.conv_bw = bw;
  g.conv_bh = bh;
  g.conv_bb = bb;
  cudaStream_t s = (cudaStream_t)stream;
  const int bn = N <= 32 ? 32 : N <= 64 ? 64 : 128;
  return bn == 32 ? conv_tcp_bn<32>(g, X, B, cs, s)
         : bn == 64 ? conv_tcp_bn<64>(g, X, B, cs, s)
                    : conv_tcp_bn<128>(g, X, B, cs, s);
}

ddflb_status ddflb_nn_set_conv_path(int32_t path) {
  if (path < 0 || path > 1) return bad("set_conv_path: path must be 0 or 1");
  g_conv_path = path;
  return DDFLB_OK;
}

ddflb_status ddflb_nn_conv3x3_flip(const void* Wt, int32_t Co, int32_t Ci, void* Wf,
                                   void* stream) {
  if (!Wt || !Wf || Co <= 0 || Ci <= 0) return bad("conv3x3_flip: bad arguments");
  const int64_t n = (int64_t)Co * 9 * Ci;
  k_conv_flip<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16*)Wt, Co, Ci, (bf16*)Wf);
  return launched("conv3x3_flip");
}

ddflb_status ddflb_nn_im2col(const void* X, int32_t B, int32_t H, int32_t W, int32_t C,
                             int32_t cs, void* col, int32_t transposed, void* stream) {
  if (!X || !col || B <= 0 || H <= 0 || W <= 0 || C <= 0 || cs < C) return bad("im2col: bad args");
  const int64_t n = (int64_t)B * H * W * 9 * C;
  cudaStream_t st = (cudaStream_t)stream;
  const bool v8 = C % 8 == 0 && cs % 8 == 0 && (uintptr_t)X % 16 == 0 && (uintptr_t)col % 16 == 0;
  if (v8) {
    if (transposed)
      k_im2col_t_v8<<<grid_for(n / 8), 256, 0, st>>>((const bf16*)X, B, H, W, C / 8, cs,
                                                     (bf16*)col);
    else if (!transposed)
      k_im2col_v8<<<grid_for(n / 8), 256, 0, st>>>((const bf16*)X, B, H, W, C / 8, cs,
                                                   (bf16*)col);
  } else if (transposed) {
    k_im2col_t<<<grid_for(n), 256, 0, st>>>((const bf16*)X, B, H, W, C, cs, (bf16*)col);
  } else {
    k_im2col<<<grid_for(n), 256, 0, st>>>((const bf16*)X, B, H, W, C, cs, (bf16*)col);
  }
  return launched("im2col");
}

ddflb_status ddflb_nn_col2im(const float* dcol, int32_t B, int32_t H, int32_t W, int32_t C,
                             float* dX, int32_t cs, void* stream) {
  if (!dcol || !dX || B <= 0 || H <= 0 || W <= 0 || C <= 0 || cs < C) return bad("col2im: bad args");
  const int64_t n = (int64_t)B * H * W * C;
  if (C % 4 == 0 && cs % 4 == 0 && (uintptr_t)dcol % 16 == 0 && (uintptr_t)dX % 16 == 0)
    k_col2im_v4<<<grid_for(n / 4), 256, 0, (cudaStream_t)stream>>>(dcol, B, H, W, C / 4, dX, cs);
  else
    k_col2im<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(dcol, B, H, W, C, dX, cs);
  return launched("col2im");
}

ddflb_status ddflb_nn_transpose(const void* src, int32_t M, int32_t N, int32_t lds, void* dst,
                                void* stream) {
  if (!src || !dst || M <= 0 || N <= 0 || lds < N) return bad("transpose: bad args");
  dim3 grid((N + 31) / 32, (M + 31) / 32), block(32, 8);
  k_transpose<<<grid, block, 0, (cudaStream_t)stream>>>((const bf16*)src, M, N, lds, (bf16*)dst);
  return launched("transpose");
}

ddflb_status ddflb_nn_pool(const void* X, int32_t B, int32_t H, int32_t W, int32_t C, int32_t csx,
                           void* Y, int32_t csy, void* stream) {
  if (!X || !Y || H % 2 || W % 2 || C <= 0) return bad("pool: bad args");
  const int64_t n = (int64_t)B * (H / 2) * (W / 2) * C;
  k_pool<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16*)X, B, H, W, C, csx,
                                                        (bf16*)Y, csy);
  return launched("pool");
}

ddflb_status ddflb_nn_pool_bwd(const float* dY, int32_t B, int32_t H, int32_t W, int32_t C,
                               int32_t csy, float* dX, int32_t csx, int32_t accumulate,
                               void* stream) {
  if (!dY || !dX || H % 2 || W % 2 || C <= 0) return bad("pool_bwd: bad args");
  const int64_t n = (int64_t)B * H * W * C;
  k_pool_bwd<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(dY, B, H, W, C, csy, dX, csx,
                                                            accumulate);
  return launched("pool_bwd");
}

ddflb_status ddflb_nn_upsample(const void* X, int32_t B, int32_t H, int32_t W, int32_t C,
                               int32_t csx, void* Y, int32_t csy, void* stream) {
  if (!X || !Y || C <= 0) return bad("upsample: bad args");
  const int64_t n = (int64_t)B * 4 * H * W * C;
  k_upsample<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16*)X, B, H, W, C, csx,
                                                            (bf16*)Y, csy);
  return launched("upsample");
}

ddflb_status ddflb_nn_upsample_bwd(const float* dY, int32_t B, int32_t H, int32_t W, int32_t C,
                                   int32_t csy, float* dX, int32_t csx, void* stream) {
  if (!dY || !dX || C <= 0) return bad("upsample_bwd: bad args");
  const int64_t n = (int64_t)B * H * W * C;
  k_upsample_bwd<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(dY, B, H, W, C, csy, dX, csx);
  return launched("upsample_bwd");
}

ddflb_status ddflb_nn_act_bwd(float* g, const void* y, int64_t rows, int32_t C, int32_t csg,
                              int32_t csy, int32_t act, void* gb, int32_t csb, void* stream) {
  if (!g || !y || rows <= 0 || C <= 0) return bad("act_bwd: bad args");
  k_act_bwd<<<grid_for(rows * C), 256, 0, (cudaStream_t)stream>>>(g, (const bf16*)y, rows, C, csg,
                                                                  csy, act, (bf16*)gb, csb);
  return launched("act_bwd");
}

ddflb_status ddflb_nn_bias_grad(const float* g, int64_t rows, int32_t C, int32_t cs, float* db,
                                void* stream) {
  if (!g || !db || rows <= 0 || C <= 0) return bad("bias_grad: bad args");
  cudaStream_t st = (cudaStream_t)stream;
  if (C <= kBiasMaxC && rows >= 4096) {
    // the scratch is one per process: calls on different streams must not overlap
    dim3 grid((C + 31) / 32, kBiasChunks);
    k_bias_grad_part<<<grid, 256, 0, st>>>(g, rows, C, cs);
    k_bias_grad_final<<<(C + 127) / 128, 128, 0, st>>>(C, kBiasChunks, db);
  } else {
    k_bias_grad<<<C, 256, 0, st>>>(g, rows, C, cs, db);
  }
  return launched("bias_grad");
}

ddflb_status ddflb_nn_mse(const float* pred, const float* target, int64_t n, float* grad,
                          double* dev_partial, double* dev_loss, void* stream) {
  if (!pred || !target || !dev_partial || !dev_loss || n <= 0) return bad("mse: bad args");
  const int nb = 256;  // dev_partial holds 256 doubles
  k_mse<<<nb, 256, 0, (cudaStream_t)stream>>>(pred, target, n, grad, dev_partial);
  k_sum<<<1, 32, 0, (cudaStream_t)stream>>>(dev_partial, nb, 1.0 / (double)n, dev_loss);
  return launched("mse");
}

ddflb_status ddflb_nn_adam(float* w, const float* g, float* m, float* v, void* wb, int64_t n,
                           float lr, float beta1, float beta2, float eps, int64_t t, float wd,
                           void* stream) {
  if (!w || !g || !m || !v || n <= 0 || t < 1) return bad("adam: bad args");
  const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
  k_adam<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(w, g, m, v, (bf16*)wb, n, lr, beta1,
                                                         beta2, eps, c1, c2, wd);
  return launched("adam");
}

ddflb_status ddflb_nn_cast_bf16(const float* x, int64_t rows, int32_t C, int32_t csx, void* y,
                                int32_t csy, void* stream) {
  if (!x || !y || rows <= 0 || C <= 0) return bad("cast: bad args");
  k_cast_bf16<<<grid_for(rows * C), 256, 0, (cudaStream_t)stream>>>(x, rows, C, csx, (bf16*)y,
                                                                    csy);
  return launched("cast");
}

}  // extern "C"
