// Periodic 3x3 convolutions with 32 input channels on the 5th-generation tensor cores
// (tcgen05): implicit GEMM over M = 128 output pixels (one row segment of one image)
// and K = 9 taps x 32 input channels, BF16 operands in shared memory, FP32
// accumulators in tensor memory (TMEM).
//
// Row-stacked weights: input row r contributes to output rows r+1, r, r-1 through the
// weight taps dy = 0, 1, 2.  The B operand stacks, for each dx and 16-channel K-step,
// the three dy blocks of NB output channels (NB = 32, or 16 for the one-channel guess
// layer) along N, so one MMA of N = 3 NB applies an input plane to all three output
// rows at once: 6 MMAs per input row instead of 18 per output row, each reading the
// 128-row A window once for three times the work.  Output rows accumulate in a ring
// of kBlocks TMEM blocks of NB columns; the epilogue zeroes a block after reading it,
// so every MMA accumulates.  An MMA whose output rows would wrap the ring is split in
// two, and at the ends of a run only the rows inside the run are computed.
//
// A operand: the K-major layout with 64-byte swizzle.  A pixel (32 channels, 64 bytes)
// is one row; 16-byte chunk c of the row at shared address a is stored at chunk
// c ^ ((a >> 7) & 3), the pattern TMA applies when it writes a 64-byte-swizzled box
// (the MMA unit derives the pattern from the same absolute address bits).  An input
// row segment (pixels x0-1 .. x0+128 of one image row, periodic) is one "plane" of 130
// consecutive pixel rows; a tap (dy, dx) is the 128-row window starting at pixel dx of
// the plane of input row y-1+dy, i.e. a 64*dx-byte change of the descriptor's start
// address, and the two K-steps of 16 channels are a further 32-byte offset.  The
// weights (B) are staged once per CTA in the same 64-byte-swizzled K-major form, one
// row of 32 input channels per (dx, stacked output channel).
//
// Work order: the tiles of an image are numbered strip by strip (a strip = the tiles
// of one 128-pixel column range, y = 0 .. H-1) and each CTA takes one contiguous range
// of that order.  Consecutive tiles of a run down a strip share two of their three
// input planes, so the planes live in a ring of kSlots shared-memory slots and each
// tile after the first of a run loads only its new row y+1: one 8 KB TMA box per tile.
//
// Warp roles of the persistent kernel (one CTA per SM):
//   warp 0      producer: walks the CTA's plane loads in order; per load one TMA
//               tensor load (the 128 body pixels, 8 KB contiguous in global memory)
//               and the two periodic halo pixels with cp.async, completing on the
//               slot's full barrier;
//   warp 1      one thread walks the input rows: per row the 6 MMAs (3 dx x 2 K-steps)
//               into the ring blocks of the output rows it touches, then commits them
//               to the barriers that free the plane and publish the output row the
//               row completes;
//   warps 2..17 epilogue, two groups of 8 warps on alternate tiles: warp w reads
//               TMEM lanes 32 (w % 4) .. +31 (one pixel per thread) and 16 of the
//               block's columns, zeroes them, applies the epilogue, and stages the
//               tile's outputs in shared memory in their global (NHWC) order; one
//               thread of the group writes the tile back with bulk asynchronous
//               copies (a tile's outputs are one contiguous block).
// All mbarrier waits are bounded; a wait that gives up raises an abort flag that
// every role checks, and sets the device flag read by mpfc_cnn_tensor_path_status.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include "../../include/mpfc.h"
#include "../../include/mpfc_cnn.h"
#include "cnn_math.cuh"
#include "mpfc_internal.h"

namespace {

constexpr int kTM = 128;                    // pixels per tile (TMEM lanes)
constexpr int kCin = 32;
constexpr int kChunks = kCin / 8;           // 8-channel (16-byte) chunks of a pixel
constexpr int kPixBytes = kCin * 2;         // one pixel row of the A operand
constexpr int kSlotBytes = 9 * 1024;        // one plane slot (130 pixels used)
constexpr int kPlaneLead = 1024 - kPixBytes;   // pixel p = 1 (first body pixel) lands 1024-byte aligned
constexpr int kSlots = 12;                  // plane ring: 3 in use by a tile + 9 loads of look-ahead
constexpr int kTxBytes = kTM * kPixBytes;   // TMA bytes per plane load
constexpr int kHaloLanes = 2 * kChunks;     // (side, chunk) cp.async copies per plane
constexpr int kBBytes = 3 * 96 * kPixBytes;     // 3 dx x 96 stacked output rows x 64 bytes
constexpr int kBlocks = 16;                 // TMEM ring of output-row accumulators
constexpr int kOutBf16 = kTM * 32 * 2, kOutF32 = kTM * 32 * 4;
constexpr int kOutBytes = kOutBf16 + kOutF32;
constexpr int kEpiWarps = 16;               // 4 lane quarters x 4 groups of 8 columns
constexpr int kThreads = 64 + 32 * kEpiWarps;
// shared-memory map (offsets from a 1024-byte aligned base)
constexpr int kOffA = 0;
constexpr int kOffB = kOffA + kSlots * kSlotBytes + 1024;   // the last slot's halo pixel spills 64 bytes
constexpr int kOffOut = kOffB + kBBytes;
constexpr int kOffBias = kOffOut + 2 * kOutBytes;
constexpr int kOffBar = kOffBias + 32 * 4;  // full[kSlots], empty[kSlots], accfull[kBlocks], accempty[kBlocks]
constexpr int kOffMisc = kOffBar + (2 * kSlots + 2 * kBlocks) * 8;   // TMEM address, abort flag
constexpr int kSmem = kOffMisc + 16 + 1024;
static_assert(kPlaneLead + 130 * kPixBytes <= kSlotBytes + kPlaneLead, "plane layout");
static_assert(kSlotBytes % 1024 == 0 && kOffB % 1024 == 0 && kOffOut % 1024 == 0, "alignment");
static_assert(kSmem <= 227 * 1024, "shared memory");
constexpr long long kSpinLimit = 200000000ll;   // clock cycles (about 0.1 s) per wait, by default

// Epilogue modes (same meaning as the mma.sync kernel's).
constexpr int kModeGelu = 0, kModeLinear = 1, kModeGeluGrad = 2, kModeGuess = 3;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (SM100 format): start address, leading- and
// stride-dimension byte offsets (all >> 4), descriptor version 1, layout type
// (0 = no swizzle, 4 = 64-byte swizzle).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout = 0) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)(layout & 7u) << 61;
  return d;
}

// Instruction descriptor of kind::f16: D in F32, A and B in BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Set to 1 by a CTA whose wait gave up; read and cleared by mpfc_cnn_tensor_path_status.
__device__ int g_tc_fail = 0;
// The wait limit in clock cycles, and the failure-injection switch of the test hook
// (mpfc_cnn_test_withhold_load): when set, CTA 0 skips the tensor copy of its first
// input row, so that the MMA issuer's wait on that row runs out.
__device__ long long g_tc_spin_limit = kSpinLimit;
__device__ int g_tc_withhold = 0;

// Bounded wait on an mbarrier phase; false if the CTA aborts (this wait timed out, or
// another role's did).
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  const long long t0 = clock64(), limit = g_tc_spin_limit;
  while (true) {
    if (try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      atomicExch(&g_tc_fail, 1);
      return false;
    }
  }
}

// Bounded wait that ignores the abort flag: the drains before a CTA exits, which wait
// for asynchronous copies and MMAs already issued (false if the limit ran out).
__device__ __forceinline__ bool drain_bar(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64(), limit = g_tc_spin_limit;
  while (!try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

struct TcArgs {
  const __nv_bfloat16* x;   // [B][H][W][32] (also described by the tensor map)
  const __nv_bfloat16* wk;  // [cout_p][288] packed (k = tap * 32 + c)
  const float* bias;        // [cout] (nullable)
  int B, H, W, cout, cout_p, mode;
  __nv_bfloat16* y_bf16;    // [B][H][W][32] (modes 0, 2)
  float* y_f32;             // [B][H][W][32] (modes 1, 2)
  float* z_f32;             // mode 0: saved pre-activation (nullable); mode 2: gelu input of the layer below
  double* phi0;             // mode 3: [H][W] field the scaled output channel 0 is added to
  double scale;
};

// Tile t of the strip-major order -> image b, tile row y, column offset x0.
struct TileOrder {
  int H, tiles_x;
  __device__ __forceinline__ void decode(int t, int& b, int& y, int& x0) const {
    const int per_img = H * tiles_x;
    b = t / per_img;
    const int rem = t - b * per_img;
    const int strip = rem / H;
    y = rem - strip * H;
    x0 = strip * kTM;
  }
  // whether tile t + 1 continues t's run down the same strip
  __device__ __forceinline__ bool continues(int t) const { return (t + 1) % H != 0; }
};

template <int NB>
__global__ void __launch_bounds__(kThreads, 1) k_conv3x3_tc(const __grid_constant__ CUtensorMap tmap, TcArgs A) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const uint32_t sbase = smem_addr(smem);
  float* bias_s = reinterpret_cast<float*>(smem + kOffBias);
  const uint32_t bar0 = sbase + kOffBar;
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (kSlots + s); };
  auto accfull = [&](int j) { return bar0 + 8u * (2 * kSlots + j); };
  auto accempty = [&](int j) { return bar0 + 8u * (2 * kSlots + kBlocks + j); };
  auto plane = [&](int slot) { return sbase + kOffA + (uint32_t)(slot * kSlotBytes + kPlaneLead); };   // pixel 0
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kOffMisc + 4);
  const uint32_t drain = sbase + kOffMisc + 8;   // the MMA issuer's final commit
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 1) {   // TMEM: the ring of kBlocks output-row blocks of NB columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(kBlocks * NB));   // the same count is freed at the end
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < kSlots; ++s) {
      bar_init(full(s), 1 + kHaloLanes);   // lane 0's expect_tx arrival + the halo cp.async arrivals
      bar_init(empty(s), 1);
    }
    for (int j = 0; j < kBlocks; ++j) {
      bar_init(accfull(j), 1);
      bar_init(accempty(j), kEpiWarps / 2);   // the 8 warps of the group that reads the block
    }
    bar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
  }
  if (tid < 32) bias_s[tid] = (A.bias && tid < A.cout) ? A.bias[tid] : 0.f;
  // stacked weights, K-major with 64-byte swizzle like A: row (dx, n), n = sb NB + co,
  // holds the 32 input channels of tap (dy = 2 - sb, dx) for output channel co (zero
  // past cout_p); its 16-byte chunk cc sits at chunk cc ^ ((row address >> 7) & 3)
  const uint4* wg = reinterpret_cast<const uint4*>(A.wk);
  for (int t = tid; t < 3 * 3 * NB * kChunks; t += kThreads) {
    const int cc = t & 3, row = t >> 2, dx = row / (3 * NB), n = row % (3 * NB);
    const int sb = n / NB, co = n % NB, tap = (2 - sb) * 3 + dx;
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    if (co < A.cout_p) w = wg[(size_t)co * (9 * kCin / 8) + tap * kChunks + cc];
    const uint32_t ra = (uint32_t)(kOffB + row * kPixBytes);   // kOffB is 1024-byte aligned, as is sbase
    *reinterpret_cast<uint4*>(smem + ra + ((cc ^ ((ra >> 7) & 3)) << 4)) = w;
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  if (warp >= 2 && warp < 10 && ((warp - 2) >> 2) * 16 < NB) {
    // zero the ring: warp w of the first epilogue group owns lanes 32 (w % 4).. and the
    // 16 columns of half (w - 2) / 4 of every block
    const uint32_t zero = 0u;
    for (int j = 0; j < kBlocks; ++j) {
      const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(j * NB + ((warp - 2) >> 2) * 16);
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
          "r"(zero)
          : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");

  const TileOrder order{A.H, A.W / kTM};
  const int ntiles = A.B * A.H * order.tiles_x;   // the host keeps this below 2^30
  const int t_begin = (int)((long long)blockIdx.x * ntiles / gridDim.x);
  const int t_end = (int)((long long)(blockIdx.x + 1) * ntiles / gridDim.x);

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    // Plane loads in order: a run's first tile loads rows y-1, y, y+1, every later tile
    // of the run row y+1; load k goes to slot k % kSlots once the load kSlots earlier
    // has been released.  Lanes 0..7 copy the two periodic halo pixels (side, chunk)
    // with cp.async, completing on the slot's full barrier; lane 0 adds the TMA box.
    // Nothing here waits on memory, so the producer runs ahead by the whole ring.
    const char* xg = reinterpret_cast<const char*>(A.x);
    const int hside = lane >> 2, hq = lane & 3;
    const bool withhold = g_tc_withhold != 0 && blockIdx.x == 0;   // test hook: skip load 0's tensor copy
    int k = 0;
    for (int t = t_begin; t < t_end; ++t) {
      int b, y, x0;
      order.decode(t, b, y, x0);
      const bool first = t == t_begin || !order.continues(t - 1);
      for (int r = first ? 0 : 2; r < 3; ++r, ++k) {
        const int s = k % kSlots, use = k / kSlots;
        bool ok = use == 0 || wait_bar(empty(s), (uint32_t)((use - 1) & 1), abort_flag);
        if (!__all_sync(0xffffffffu, ok)) break;
        int gy = y + r - 1;
        gy = gy < 0 ? gy + A.H : (gy >= A.H ? gy - A.H : gy);
        const uint32_t pl = plane(s);
        if (lane < kHaloLanes) {
          const int gx = hside ? (x0 + kTM == A.W ? 0 : x0 + kTM) : (x0 == 0 ? A.W - 1 : x0 - 1);
          const char* src = xg + ((((size_t)b * A.H + gy) * A.W + gx) * kChunks + hq) * 16;
          const uint32_t px = pl + (uint32_t)((hside ? 129 : 0) * kPixBytes);
          const uint32_t dst = px + (uint32_t)((hq ^ ((px >> 7) & 3)) << 4);   // 64-byte swizzle
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
          asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(full(s)) : "memory");
        }
        if (lane == 0 && !(withhold && k == 0)) {
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full(s)), "r"(kTxBytes)
                       : "memory");
          asm volatile(
              "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(pl + kPixBytes),   // 1024-byte aligned
              "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(0), "r"(x0), "r"(b * A.H + gy), "r"(full(s))
              : "memory");
        }
      }
      if (*abort_flag) break;
    }
    // Drain before the CTA exits: this lane's halo copies, then (lane 0) the tensor
    // copies of the last kSlots loads, which an aborted MMA issuer may not have waited
    // for.  A load whose phase already completed returns at once; the load the test hook
    // withheld never completes and is skipped.
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (lane == 0)
      for (int kk = k > kSlots ? k - kSlots : 0; kk < k; ++kk)
        if (!(withhold && kk == 0)) drain_bar(full(kk % kSlots), (uint32_t)((kk / kSlots) & 1));
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t b0 = sbase + kOffB;
      int k = 0;   // plane loads consumed
      bool ok = true;
      for (int ts = t_begin; ts < t_end && ok;) {
        int te = ts;   // the run ts .. te down one strip
        while (te + 1 < t_end && order.continues(te)) ++te;
        const int n = te - ts + 1, i_s = ts - t_begin;
        for (int rr = -1; rr <= n; ++rr, ++k) {   // input row y0 + rr (output rows rr-1, rr, rr+1 of the run)
          const int s = k % kSlots;
          ok = wait_bar(full(s), (uint32_t)((k / kSlots) & 1), abort_flag);
          if (ok && rr + 1 <= n - 1) {   // first contribution to output row rr + 1: its block must be free
            const int i = i_s + rr + 1;
            if (i >= kBlocks)
              ok = wait_bar(accempty(i % kBlocks), (uint32_t)(((i / kBlocks) - 1) & 1), abort_flag);
          }
          if (!ok) break;
          // the halo chunks arrived through cp.async (generic proxy); the MMAs read
          // through the async proxy
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int qa = rr - 1 > 0 ? rr - 1 : 0, qb = rr + 1 < n - 1 ? rr + 1 : n - 1;
          const int cnt = qb - qa + 1;                 // 1 .. 3 output rows
          const int ja = (i_s + qa) % kBlocks;         // ring block of output row qa
          const int sba = qa - rr + 1;                 // its block in the weight stack (dy = 2 - sba)
          const int c1 = cnt < kBlocks - ja ? cnt : kBlocks - ja;
          const uint32_t pl = plane(s);
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              const uint64_t ad = make_desc(pl + (uint32_t)(dx * kPixBytes + kk * 32), 16, 8 * kPixBytes, 4);
              const uint32_t bb = b0 + (uint32_t)(dx * 3 * NB * kPixBytes + kk * 32);
              const uint64_t bd = make_desc(bb + (uint32_t)(sba * NB * kPixBytes), 16, 8 * kPixBytes, 4);
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, 1, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(ja * NB)),
                  "l"(ad), "l"(bd), "r"(idesc(c1 * NB)));
              if (c1 < cnt) {   // the rows past the ring's end continue at block 0
                const uint64_t bd2 = make_desc(bb + (uint32_t)((sba + c1) * NB * kPixBytes), 16, 8 * kPixBytes, 4);
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, 1, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd2), "r"(idesc((cnt - c1) * NB)));
              }
            }
          }
          mma_commit(empty(s));                                            // the plane is used once
          if (rr - 1 >= 0) mma_commit(accfull((i_s + rr - 1) % kBlocks));  // output row rr - 1 is complete
        }
        ts = te + 1;
      }
      // every MMA issued has completed before the tensor memory is freed (also after an abort)
      mma_commit(drain);
      drain_bar(drain, 0u);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    // Two groups of 8 warps take alternate tiles (group G the tiles i = G mod 2), so one
    // group's GELU math overlaps the other's stores and barriers.  Within a group, warp w
    // reads lane quarter w % 4 and the 16 columns of half h of the block.
    const int e = warp - 2, grp = e >> 3, qd = warp & 3, h = (e >> 2) & 1;
    const bool owns_cols = h * 16 < NB;
    const bool leader = (e & 7) == 0 && lane == 0;        // issues the group's bulk copies
    const int p = qd * 32 + lane;                         // this thread's pixel in the tile
    const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
    const float* bias_h = bias_s + (16 * h & 31);   // this half's 16 biases (shared-memory broadcast)
    const bool f32_out = A.mode == kModeLinear || A.mode == kModeGeluGrad || A.z_f32 != nullptr;
    unsigned char* ob = smem + kOffOut + grp * kOutBytes;  // this group's stage buffer
    int b = 0, y = 0, x0 = 0;   // tile t of the order, advanced by two tiles per iteration (no divisions)
    if (t_begin + grp < t_end) order.decode(t_begin + grp, b, y, x0);
    for (int i = grp, t = t_begin + grp; t < t_end; t += 2, i += 2) {
      const int blk = i % kBlocks;
      const size_t pix0 = ((size_t)b * A.H + y) * A.W + x0;
      for (y += 2; y >= A.H;) {   // strip-major: down the strip, then the next strip, then the next image
        y -= A.H;
        x0 += kTM;
        if (x0 >= A.W) {
          x0 = 0;
          ++b;
        }
      }
      float4 zin[4];
      if (A.mode == kModeGeluGrad) {
        const float4* zg = reinterpret_cast<const float4*>(A.z_f32 + (pix0 + p) * 32 + h * 16);
#pragma unroll
        for (int v = 0; v < 4; ++v) zin[v] = zg[v];
      }
      bool ok = wait_bar(accfull(blk), (uint32_t)((i / kBlocks) & 1), abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      asm volatile("tcgen05.fence::after_thread_sync;");
      uint32_t r[16];
      if (ok && owns_cols) {
        // read this warp's 16 columns of the block, then zero them for the block's next row
        const uint32_t taddr = tmem + lane_base + (uint32_t)(blk * NB + h * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const uint32_t zero = 0u;
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(
                taddr),
            "r"(zero)
            : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) bar_arrive(accempty(blk));   // this warp's share of the block is read and zeroed
      if (A.mode == kModeGuess) {
        if (ok && h == 0) A.phi0[pix0 + p] += A.scale * (double)(__uint_as_float(r[0]) + bias_h[0]);
        continue;
      }
      float o[16];
      if (A.mode == kModeGeluGrad) {
        const float* zz = reinterpret_cast<const float*>(zin);
#pragma unroll
        for (int c = 0; c < 16; ++c)
          o[c] = 16 * h + c < A.cout ? __uint_as_float(r[c]) * mpfc_cnn_math::gelu_grad(zz[c]) : 0.f;
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) o[c] = 16 * h + c < A.cout ? __uint_as_float(r[c]) + bias_h[c] : 0.f;
      }
      float q[16];
      if (A.mode == kModeGelu) {
        float zb[8], gb[8];
#pragma unroll
        for (int half = 0; half < 2; ++half) {
#pragma unroll
          for (int c = 0; c < 8; ++c) zb[c] = o[8 * half + c];
          mpfc_cnn_math::gelu8(zb, gb);
#pragma unroll
          for (int c = 0; c < 8; ++c) q[8 * half + c] = 16 * h + 8 * half + c < A.cout ? gb[c] : 0.f;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) q[c] = o[c];
      }
      // this group's stage buffer must have been read by its previous bulk copy
      if (leader) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      asm volatile("bar.sync %0, 256;" ::"r"(1 + grp) : "memory");
      if (ok) {
        if (f32_out) {
          uint4* d = reinterpret_cast<uint4*>(ob + kOutBf16 + p * 128 + h * 64);
#pragma unroll
          for (int v = 0; v < 4; ++v)
            d[v] = make_uint4(__float_as_uint(o[4 * v]), __float_as_uint(o[4 * v + 1]), __float_as_uint(o[4 * v + 2]),
                              __float_as_uint(o[4 * v + 3]));
        }
        if (A.mode != kModeLinear) {
          uint4* d = reinterpret_cast<uint4*>(ob + p * 64 + h * 32);
          d[0] = make_uint4(pack_bf16(q[0], q[1]), pack_bf16(q[2], q[3]), pack_bf16(q[4], q[5]), pack_bf16(q[6], q[7]));
          d[1] = make_uint4(pack_bf16(q[8], q[9]), pack_bf16(q[10], q[11]), pack_bf16(q[12], q[13]),
                            pack_bf16(q[14], q[15]));
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("bar.sync %0, 256;" ::"r"(1 + grp) : "memory");
      if (leader && !*abort_flag) {
        if (f32_out) {
          float* dst = (A.mode == kModeGelu ? A.z_f32 : A.y_f32) + pix0 * 32;
          asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                       "r"(smem_addr(ob + kOutBf16)), "r"(kOutF32)
                       : "memory");
        }
        if (A.mode != kModeLinear) {
          __nv_bfloat16* dst = A.y_bf16 + pix0 * 32;
          asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(ob)),
                       "r"(kOutBf16)
                       : "memory");
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
    if (leader) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBlocks * NB));
}

int g_use_tc = 1;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

// Tensor map of the input activations viewed as [B*H rows][W pixels][32 channels]
// bf16, box = 32 channels x 128 pixels x 1 row (8 KB contiguous), 64-byte swizzle.
int make_tmap(CUtensorMap* map, const void* x, int B, int H, int W) {
  {
    std::lock_guard<std::mutex> lk(g_encode_mu);
    if (!g_encode) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
      if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        mpfc_set_cuda_error(e != cudaSuccess ? e : cudaErrorSymbolNotFound, "cuTensorMapEncodeTiled", __FILE__,
                            __LINE__);
        return MPFC_ERR_CUDA;
      }
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
  }
  cuuint64_t dims[3] = {(cuuint64_t)kCin, (cuuint64_t)W, (cuuint64_t)B * H};
  cuuint64_t strides[2] = {(cuuint64_t)kCin * 2, (cuuint64_t)W * kCin * 2};
  cuuint32_t box[3] = {(cuuint32_t)kCin, (cuuint32_t)kTM, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(x), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? MPFC_OK : MPFC_ERR_INVALID;
}

template <int NB>
int launch_tc(const CUtensorMap& map, const TcArgs& A, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) {
      mpfc_set_cuda_error(e, "tc conv smem", __FILE__, __LINE__);
      return MPFC_ERR_CUDA;
    }
    attr = true;
  }
  const long long ntiles = (long long)A.B * A.H * (A.W / kTM);
  const long long sms = mpfc::sm_count();
  const int grid = (int)(ntiles < sms ? ntiles : sms);   // persistent: one CTA per SM
  k_conv3x3_tc<NB><<<grid, kThreads, kSmem, s>>>(map, A);
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
  if ((reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(wk) & 15) ||
      (reinterpret_cast<uintptr_t>(y_bf16) & 15) || (reinterpret_cast<uintptr_t>(y_f32) & 15) ||
      (reinterpret_cast<uintptr_t>(z_f32) & 15))
    return MPFC_ERR_INVALID;   // 16-byte vector and bulk copies
  if ((long long)B * H * (W / kTM) >= (1ll << 30)) return MPFC_ERR_INVALID;   // tile indices stay 32-bit
  CUtensorMap map;
  int rc = make_tmap(&map, x, B, H, W);
  if (rc != MPFC_OK) return rc;
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
  return mode == kModeGuess ? launch_tc<16>(map, A, s) : launch_tc<32>(map, A, s);
}

extern "C" int mpfc_cnn_set_tensor_path(int use_tcgen05) {
  g_use_tc = use_tcgen05 ? 1 : 0;
  return MPFC_OK;
}

extern "C" int mpfc_cnn_test_withhold_load(int withhold, long long spin_cycles) {
  if (withhold < 0 || withhold > 1 || spin_cycles < 0) return MPFC_ERR_INVALID;
  const int w = withhold;
  const long long lim = spin_cycles > 0 ? spin_cycles : kSpinLimit;
  cudaError_t e = cudaMemcpyToSymbol(g_tc_withhold, &w, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_spin_limit, &lim, sizeof(long long));
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "tc test hook", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
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
