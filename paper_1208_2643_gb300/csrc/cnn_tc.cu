// Periodic 3x3 convolutions with 32 input channels on the 5th-generation tensor cores
// (tcgen05): implicit GEMM with M = 128 output pixels (one row segment of one image),
// N = 32 (or 16) output channels, K = 9 taps x 32 input channels; BF16 operands in
// shared memory, FP32 accumulator in tensor memory (TMEM).
//
// Shared-memory operands use the canonical K-major layout without swizzle: a "core
// matrix" is 8 rows x 16 bytes (8 bf16 along K), rows 16 bytes apart, so the rows of a
// whole operand sit at a uniform 16-byte stride and a tap's pixel shift dx is just a
// 16*dx-byte offset of the descriptor's start address.  Input rows y-1, y, y+1 of the
// tile (pixels x0-1 .. x0+128, periodic) are staged as [row][8-channel chunk][pixel]
// 16-byte units; weights as [tap][chunk][out channel] 16-byte units.  One thread
// issues the 18 MMAs (9 taps x 2 K-steps of 16) and commits them to an mbarrier.
//
// Per tile the CTA overlaps the MMAs with the global loads of the next tile's input
// (held in registers), then reads the accumulator (tcgen05.ld, one pixel per thread),
// applies the epilogue, and writes the tile's outputs through a swizzled shared-memory
// stage (the A operand's space, free once the MMAs completed) so that the global
// stores are contiguous: a tile's outputs are one contiguous block of NHWC memory.
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/mpfc.h"
#include "../../include/mpfc_cnn.h"
#include "mpfc_internal.h"

namespace {

constexpr int kTM = 128;                 // pixels per tile (TMEM lanes)
constexpr int kCin = 32;
constexpr int kChunks = kCin / 8;        // 8-channel (16-byte) chunks of a pixel
constexpr int kNPix = 138;               // staged pixels per (row, chunk); 130 used, the pad spreads banks
constexpr int kUnits = 3 * 130 * kChunks;             // 16-byte units staged per tile (1560)
constexpr int kThreads = 128;
constexpr int kPerThread = (kUnits + kThreads - 1) / kThreads;   // 13
constexpr int kABytes = 3 * kChunks * kNPix * 16;     // 26496
constexpr int kBBytesMax = 9 * kChunks * 32 * 16;     // 18432
constexpr int kSmem = kABytes + kBBytesMax + 32 * 4 + 64;
static_assert(kTM * 32 * 4 + kTM * 32 * 2 <= kABytes, "output stage must fit in the A operand space");

// Epilogue modes (same meaning as the mma.sync kernel's).
constexpr int kModeGelu = 0, kModeLinear = 1, kModeGeluGrad = 2, kModeGuess = 3;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (SM100 format): start address, leading- and
// stride-dimension byte offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  return d;
}

// Instruction descriptor of kind::f16: D in F32, A and B in BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
template <int N>
__device__ __forceinline__ uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

struct TcArgs {
  const __nv_bfloat16* x;   // [B][H][W][32]
  const __nv_bfloat16* wk;  // [cout_p][288] packed (k = tap * 32 + c)
  const float* bias;        // [cout] (nullable)
  int B, H, W, cout, cout_p, mode;
  __nv_bfloat16* y_bf16;    // [B][H][W][32] (modes 0, 2)
  float* y_f32;             // [B][H][W][32] (modes 1, 2)
  float* z_f32;             // mode 0: saved pre-activation (nullable); mode 2: gelu input of the layer below
  double* phi0;             // mode 3: [H][W] field the scaled output channel 0 is added to
  double scale;
};

// Set to 1 by a CTA whose MMA-completion wait gave up; read and cleared by
// mpfc_cnn_tensor_path_status.
__device__ int g_tc_fail = 0;

// Global loads of one tile's input units into registers (unit t: row r, pixel p, chunk q).
__device__ __forceinline__ void load_tile(const uint4* __restrict__ xg, const TcArgs& A, long long tile, int tiles_x,
                                          uint4 (&v)[kPerThread]) {
  const int b = (int)(tile / ((long long)A.H * tiles_x));
  const int rem = (int)(tile % ((long long)A.H * tiles_x));
  const int y = rem / tiles_x, x0 = (rem % tiles_x) * kTM;
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    const int t = threadIdx.x + i * kThreads;
    if (t < kUnits) {
      const int q = t & 3, rp = t >> 2, r = rp / 130, p = rp - r * 130;
      int gy = y + r - 1;
      gy = gy < 0 ? gy + A.H : (gy >= A.H ? gy - A.H : gy);
      int gx = x0 + p - 1;
      gx = gx < 0 ? gx + A.W : (gx >= A.W ? gx - A.W : gx);
      v[i] = __ldg(&xg[(((size_t)b * A.H + gy) * A.W + gx) * kChunks + q]);
    }
  }
}

__device__ __forceinline__ void store_tile(unsigned char* As, const uint4 (&v)[kPerThread]) {
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    const int t = threadIdx.x + i * kThreads;
    if (t < kUnits) {
      const int q = t & 3, rp = t >> 2, r = rp / 130, p = rp - r * 130;
      reinterpret_cast<uint4*>(As)[(r * kChunks + q) * kNPix + p] = v[i];
    }
  }
}

// Output stage inside the A space: fp32 [128 px][8 chunks of 4] then bf16 [128 px][4
// chunks of 8]; chunk j of pixel p sits at position j ^ (p & 7) (fp32) or
// j ^ ((p >> 1) & 3) (bf16) so that the per-pixel accesses of a warp hit distinct banks.
constexpr int kStageF32 = 0, kStageBf16 = kTM * 32 * 4;
__device__ __forceinline__ int f32_slot(int p, int j) { return p * 8 + (j ^ (p & 7)); }
__device__ __forceinline__ int bf16_slot(int p, int j) { return p * 4 + (j ^ ((p >> 1) & 3)); }

template <int N>
__global__ void __launch_bounds__(kThreads, 4) k_conv3x3_tc(TcArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* As = smem;
  unsigned char* Bs = smem + kABytes;
  float* bias_s = reinterpret_cast<float*>(smem + kABytes + kBBytesMax);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kABytes + kBBytesMax + 32 * 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kABytes + kBBytesMax + 32 * 4 + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // TMEM: 32 columns (the FP32 accumulator of 128 x N, N <= 32)
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(32));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (tid < 32) bias_s[tid] = (A.bias && tid < A.cout) ? A.bias[tid] : 0.f;
  // weights: unit (tap, q, n) = 8 channels of output row n; rows past cout_p are zero
  const uint4* wg = reinterpret_cast<const uint4*>(A.wk);
  for (int t = tid; t < 9 * kChunks * N; t += kThreads) {
    const int n = t % N, tq = t / N, tap = tq / kChunks, q = tq % kChunks;
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    if (n < A.cout_p) w = wg[(size_t)n * (9 * kCin / 8) + tap * kChunks + q];
    reinterpret_cast<uint4*>(Bs)[t] = w;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  const int tiles_x = A.W / kTM;
  const long long ntiles = (long long)A.B * A.H * tiles_x;
  const uint4* xg = reinterpret_cast<const uint4*>(A.x);
  uint4 v[kPerThread];
  if (blockIdx.x < ntiles) load_tile(xg, A, blockIdx.x, tiles_x, v);
  uint32_t phase = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int b = (int)(tile / ((long long)A.H * tiles_x));
    const int rem = (int)(tile % ((long long)A.H * tiles_x));
    const int y = rem / tiles_x, x0 = (rem % tiles_x) * kTM;
    const size_t pix0 = ((size_t)b * A.H + y) * A.W + x0;
    store_tile(As, v);
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_addr(As), b0 = smem_addr(Bs);
      int accum = 0;
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap % 3;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const uint64_t ad = make_desc(a0 + (uint32_t)(((dy * kChunks + 2 * kk) * kNPix + dx) * 16), kNPix * 16, 128);
          const uint64_t bd = make_desc(b0 + (uint32_t)(((tap * kChunks + 2 * kk) * N) * 16), N * 16, 128);
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc<N>()), "r"(accum));
          accum = 1;
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(mbar)));
    }
    // the next tile's input travels while the MMAs run
    if (tile + gridDim.x < ntiles) load_tile(xg, A, tile + gridDim.x, tiles_x, v);
    // bounded wait for the MMAs (about 50 ms of polling at most)
    uint32_t done = 0;
    const long long t0 = clock64();
    while (!done) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(smem_addr(mbar)), "r"(phase));
      if (!done && clock64() - t0 > 100000000ll) break;
    }
    // all threads take the same decision (a thread that gave up makes the block stop)
    if (__syncthreads_or(done ? 0 : 1)) {
      if (tid == 0) atomicExch(&g_tc_fail, 1);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int p = warp * 32 + lane;                    // this thread's pixel (TMEM lane)
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    if (A.mode == kModeGuess) {
      uint32_t r0;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n" : "=r"(r0) : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      A.phi0[pix0 + p] += A.scale * (double)(__uint_as_float(r0) + bias_s[0]);
    } else {
      if (A.mode == kModeGeluGrad) {
        // stage the tile's z (a contiguous block) with coalesced loads
        const uint4* zg = reinterpret_cast<const uint4*>(A.z_f32 + pix0 * 32);
        uint4* st = reinterpret_cast<uint4*>(As + kStageF32);
#pragma unroll
        for (int i = 0; i < kTM * 8 / kThreads; ++i) {
          const int u = tid + i * kThreads, pp = u >> 3, j = u & 7;
          st[f32_slot(pp, j)] = zg[u];
        }
        __syncthreads();
      }
      uint32_t r[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
          "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      float4* sf = reinterpret_cast<float4*>(As + kStageF32);
      uint4* sb = reinterpret_cast<uint4*>(As + kStageBf16);
      float o[32];
      if (A.mode == kModeGeluGrad) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4 z = sf[f32_slot(p, j)];
          o[4 * j + 0] = 4 * j + 0 < A.cout ? __uint_as_float(r[4 * j + 0]) * gelu_grad(z.x) : 0.f;
          o[4 * j + 1] = 4 * j + 1 < A.cout ? __uint_as_float(r[4 * j + 1]) * gelu_grad(z.y) : 0.f;
          o[4 * j + 2] = 4 * j + 2 < A.cout ? __uint_as_float(r[4 * j + 2]) * gelu_grad(z.z) : 0.f;
          o[4 * j + 3] = 4 * j + 3 < A.cout ? __uint_as_float(r[4 * j + 3]) * gelu_grad(z.w) : 0.f;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 32; ++c) o[c] = c < A.cout ? __uint_as_float(r[c]) + bias_s[c] : 0.f;
      }
      const bool f32_out = A.mode == kModeLinear || A.mode == kModeGeluGrad || A.z_f32 != nullptr;
      if (f32_out) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          sf[f32_slot(p, j)] = make_float4(o[4 * j], o[4 * j + 1], o[4 * j + 2], o[4 * j + 3]);
      }
      if (A.mode != kModeLinear) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float g[8];
#pragma unroll
          for (int e = 0; e < 8; ++e)
            g[e] = A.mode == kModeGelu ? (8 * j + e < A.cout ? gelu_f(o[8 * j + e]) : 0.f) : o[8 * j + e];
          sb[bf16_slot(p, j)] = make_uint4(pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), pack_bf16(g[4], g[5]),
                                           pack_bf16(g[6], g[7]));
        }
      }
      __syncthreads();
      // contiguous copy-out of the tile
      if (f32_out) {
        uint4* dst = reinterpret_cast<uint4*>((A.mode == kModeGelu ? A.z_f32 : A.y_f32) + pix0 * 32);
        const uint4* src = reinterpret_cast<const uint4*>(As + kStageF32);
#pragma unroll
        for (int i = 0; i < kTM * 8 / kThreads; ++i) {
          const int u = tid + i * kThreads, pp = u >> 3, j = u & 7;
          dst[u] = src[f32_slot(pp, j)];
        }
      }
      if (A.mode != kModeLinear) {
        uint4* dst = reinterpret_cast<uint4*>(A.y_bf16 + pix0 * 32);
        const uint4* src = reinterpret_cast<const uint4*>(As + kStageBf16);
#pragma unroll
        for (int i = 0; i < kTM * 4 / kThreads; ++i) {
          const int u = tid + i * kThreads, pp = u >> 2, j = u & 3;
          dst[u] = src[bf16_slot(pp, j)];
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();   // TMEM and the A space are free for the next tile
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32));
}

int g_use_tc = 1;

template <int N>
int launch_tc(const TcArgs& A, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) {
      mpfc_set_cuda_error(e, "tc conv smem", __FILE__, __LINE__);
      return MPFC_ERR_CUDA;
    }
    attr = true;
  }
  const long long ntiles = (long long)A.B * A.H * (A.W / kTM);
  const int grid = (int)(ntiles < 152 * 4 ? ntiles : 152 * 4);   // 4 CTAs per SM fit in shared memory
  k_conv3x3_tc<N><<<grid, kThreads, kSmem, s>>>(A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "k_conv3x3_tc", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  return MPFC_OK;
}

}  // namespace

// Whether a convolution can take the tcgen05 path: 32 input channels, 32 padded output
// channels (modes 0-2) or 8 (mode 3, one real output channel), width a multiple of 128.
bool mpfc_cnn_tc_eligible(int cin_p, int cout_p, int W, int mode) {
  if (!g_use_tc || cin_p != kCin || W % kTM != 0) return false;
  return mode == kModeGuess ? cout_p == 8 : cout_p == 32;
}

int mpfc_cnn_conv_tc(const void* x, int B, int H, int W, const void* wk, const float* bias, int cout, int cout_p,
                     int mode, void* y_bf16, float* y_f32, float* z_f32, double* phi0, double scale,
                     cudaStream_t s) {
  TcArgs A;
  A.x = (const __nv_bfloat16*)x;
  A.wk = (const __nv_bfloat16*)wk;
  A.bias = bias;
  A.B = B;
  A.H = H;
  A.W = W;
  A.cout = cout;
  A.cout_p = cout_p;
  A.mode = mode;
  A.y_bf16 = (__nv_bfloat16*)y_bf16;
  A.y_f32 = y_f32;
  A.z_f32 = z_f32;
  A.phi0 = phi0;
  A.scale = scale;
  return mode == kModeGuess ? launch_tc<16>(A, s) : launch_tc<32>(A, s);
}

extern "C" int mpfc_cnn_set_tensor_path(int use_tcgen05) {
  g_use_tc = use_tcgen05 ? 1 : 0;
  return MPFC_OK;
}

extern "C" int mpfc_cnn_tensor_path_status(void) {
  int v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_fail, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_fail, &zero, sizeof(int));
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "tc status", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  return v ? MPFC_ERR_NOT_CONVERGED : MPFC_OK;
}
