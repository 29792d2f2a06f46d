// Convolution kernels of the learned initial guess: periodic 3x3 convolutions as
// implicit GEMMs on BF16 tensor cores with FP32 accumulation (forward and data
// gradient), the weight gradient on CUDA cores with a deterministic two-pass
// reduction, the MSE loss gradient and the Adam update.
//
// Layout: activations NHWC, bf16, channels padded to CP in {4, 8, 16, 32}; images are
// periodic in x and y (the grid functions they come from are periodic).  A layer's
// weights are stored for the kernels as Wk[n][k] (bf16, k contiguous) with
// k = tap * CP_in + c_in, tap = (dy + 1) * 3 + (dx + 1), n = c_out; the FP32 master
// copy is [tap][c_in][c_out].
#include <cuda_bf16.h>
#include <math.h>

#include "../../include/mpfc.h"
#include "../../include/mpfc_cnn.h"
#include "cnn_math.cuh"
#include "mpfc_internal.h"

bool mpfc_cnn_tc_eligible(int cin_p, int cout_p, int W, int mode);
int mpfc_cnn_conv_tc(const void* x, int B, int H, int W, const void* wk, const float* bias, int cout, int cout_p,
                     int mode, void* y_bf16, float* y_f32, float* z_f32, double* phi0, double scale,
                     cudaStream_t s);

namespace {

constexpr int kTW = 32, kTH = 4;          // output tile: 32 x 4 pixels, 4 warps (one row each)
constexpr int kMaxCin = 32, kMaxCout = 32;

__device__ __forceinline__ int wrapi(int i, int n) { return ((i % n) + n) % n; }

__device__ __forceinline__ float gelu_f(float z) { return mpfc_cnn_math::gelu(z); }
__device__ __forceinline__ float gelu_grad(float z) { return mpfc_cnn_math::gelu_grad(z); }

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Epilogue modes of the forward kernel.
enum : int {
  kEpiGeluBf16 = 0,    // y = gelu(acc + bias) as bf16; z = acc + bias saved as fp32 (nullable)
  kEpiLinearF32 = 1,   // y = acc + bias as fp32
  kEpiGeluGradBf16 = 2,// dz_prev = acc * gelu'(z_prev): bf16 copy (next data gradient) and fp32 copy
  kEpiGuess = 3,       // phi0[p] += scale * (acc + bias) (fp64 field; output channel 0 only)
};

struct ConvArgs {
  const __nv_bfloat16* x;   // [B][H][W][cin_p]
  const __nv_bfloat16* wk;  // [cout_p][kpad] bf16, k = tap * cin_p + c
  const float* bias;        // [cout] (nullable)
  int B, H, W, cin_p, cout, cout_p, kpad;   // kpad: K rounded up to 16
  int mode;
  __nv_bfloat16* y_bf16;    // [B][H][W][cout_p]
  float* y_f32;             // [B][H][W][cout_p]
  float* z_f32;             // saved pre-activation (mode 0) / gelu input of the previous layer (mode 2)
  double* phi0;             // mode 3
  double scale;             // mode 3
};

// One CTA: a 32 x 4 output tile of one image, all output channels.  The input tile
// with a one-pixel periodic halo and the layer's weights are staged in shared memory;
// each warp computes one output row (two m16 tiles) against cout_p/8 n8 tiles.
__global__ void __launch_bounds__(128) k_conv3x3(ConvArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int cin = A.cin_p, KP = A.kpad, NT = A.cout_p / 8;
  const int pairs = cin / 2;
  const int ps = pairs + 4;                         // padded pixel stride in 4-byte words (bank spread)
  __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(smem);            // (kTH+2)(kTW+2) pixels
  const int xs_count = (kTH + 2) * (kTW + 2) * ps * 2;
  __nv_bfloat16* ws = xs + ((xs_count + 7) & ~7);                       // cout_p x (KP + 8)
  const int wstride = KP + 8;
  const int tid = threadIdx.x;
  const unsigned* xg = reinterpret_cast<const unsigned*>(A.x);
  unsigned* xsu = reinterpret_cast<unsigned*>(xs);
  // stage the weights once per CTA (rows of KP bf16, padded stride)
  const unsigned* wg = reinterpret_cast<const unsigned*>(A.wk);
  unsigned* wsu = reinterpret_cast<unsigned*>(ws);
  for (int t = tid; t < A.cout_p * (KP / 2); t += blockDim.x) {
    int n = t / (KP / 2), kk = t % (KP / 2);
    wsu[n * (wstride / 2) + kk] = wg[(size_t)n * (KP / 2) + kk];
  }
  const int tiles_x = (A.W + kTW - 1) / kTW, tiles_y = (A.H + kTH - 1) / kTH;
  const long long ntiles = (long long)tiles_x * tiles_y * A.B;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  const int b = (int)(tile / ((long long)tiles_x * tiles_y));
  const int trem = (int)(tile % ((long long)tiles_x * tiles_y));
  const int ty0 = (trem / tiles_x) * kTH, tx0 = (trem % tiles_x) * kTW;
  __syncthreads();   // previous tile's reads of xs are done (and the weights are staged)
  // stage the input tile (4-byte units: two channels)
  for (int t = tid; t < (kTH + 2) * (kTW + 2) * pairs; t += blockDim.x) {
    int cp = t % pairs, pix = t / pairs;
    int lx = pix % (kTW + 2), ly = pix / (kTW + 2);
    int gx = wrapi(tx0 + lx - 1, A.W), gy = wrapi(ty0 + ly - 1, A.H);
    xsu[pix * ps + cp] = xg[(((size_t)b * A.H + gy) * A.W + gx) * pairs + cp];
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, tig = lane & 3;
  const int ry = warp;                                // output row within the tile
  float acc[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
  const int ktot = 9 * cin;
  for (int k0 = 0; k0 < KP; k0 += 16) {
    // A fragments: rows = pixels (x = mt*16 + g (+8)), cols = k0 + tig*2 (+8) (+1)
    unsigned a[2][4];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      int k = k0 + tig * 2 + half * 8;
      bool valid = k < ktot;
      int tap = valid ? k / cin : 0, c = valid ? k - tap * cin : 0;
      int dy = tap / 3, dx = tap % 3;                 // 0..2 (offset + 1)
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int hi = 0; hi < 2; ++hi) {
          int px = mt * 16 + g + hi * 8;
          unsigned v = 0u;
          if (valid) v = xsu[((ry + dy) * (kTW + 2) + (px + dx)) * ps + c / 2];
          a[mt][half * 2 + hi] = v;
        }
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      if (nt >= NT) break;
      const int n = nt * 8 + g;
      unsigned bb[2];
      bb[0] = wsu[n * (wstride / 2) + (k0 + tig * 2) / 2];
      bb[1] = wsu[n * (wstride / 2) + (k0 + tig * 2 + 8) / 2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) mma_bf16_16816(acc[mt][nt], a[mt], bb);
    }
  }
  // epilogue: acc[mt][nt][e] is (pixel mt*16 + g + 8*(e>>1), channel nt*8 + tig*2 + (e&1))
  const int oy = ty0 + ry;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      if (nt >= NT) break;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int px = tx0 + mt * 16 + g + 8 * (e >> 1);
        int co = nt * 8 + tig * 2 + (e & 1);
        if (oy >= A.H || px >= A.W) continue;
        size_t pix = ((size_t)b * A.H + oy) * A.W + px;
        float v = acc[mt][nt][e];
        if (A.mode == kEpiGeluBf16) {
          float z = co < A.cout ? v + (A.bias ? A.bias[co] : 0.f) : 0.f;
          if (A.z_f32) A.z_f32[pix * A.cout_p + co] = z;
          A.y_bf16[pix * A.cout_p + co] = __float2bfloat16_rn(co < A.cout ? gelu_f(z) : 0.f);
        } else if (A.mode == kEpiLinearF32) {
          A.y_f32[pix * A.cout_p + co] = co < A.cout ? v + (A.bias ? A.bias[co] : 0.f) : 0.f;
        } else if (A.mode == kEpiGeluGradBf16) {
          float d = co < A.cout ? v * gelu_grad(A.z_f32[pix * A.cout_p + co]) : 0.f;
          A.y_f32[pix * A.cout_p + co] = d;
          A.y_bf16[pix * A.cout_p + co] = __float2bfloat16_rn(d);
        } else {
          if (co == 0) A.phi0[pix] += A.scale * (double)(v + (A.bias ? A.bias[0] : 0.f));
        }
      }
    }
  }   // tile loop
}

// Weight gradient of one tap for a chunk of pixels:
//   dW[tap][ci][co] += sum_p x[p + off(tap)][ci] dz[p][co],
// CTA (tap, chunk) writes its partial to part[chunk][tap][ci][co]; db likewise from the
// centre tap's CTAs.  256 threads, each owning (ci, co) pairs ci = t/8.., co = ...
constexpr int kWgChunk = 2048;
__global__ void __launch_bounds__(256) k_wgrad_partial(const __nv_bfloat16* __restrict__ x, const float* __restrict__ dz,
                                                       int B, int H, int W, int cin_p, int cin, int cout_p, int cout,
                                                       float* __restrict__ part, float* __restrict__ dbpart) {
  const int tap = blockIdx.y, chunk = blockIdx.x;
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  const long long npix = (long long)B * H * W;
  const long long p0 = (long long)chunk * kWgChunk;
  __shared__ float xs[64][kMaxCin];
  __shared__ float ds[64][kMaxCout];
  const int tid = threadIdx.x;
  // thread owns pairs (ci, co) with ci = tid / 8 (0..31), co = (tid % 8) * 4 + 0..3
  const int ci = tid >> 3, co0 = (tid & 7) * 4;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float dbacc = 0.f;
  for (long long base = p0; base < p0 + kWgChunk && base < npix; base += 64) {
    __syncthreads();
    for (int t = tid; t < 64 * kMaxCin; t += 256) {
      int pp = t / kMaxCin, c = t % kMaxCin;
      long long p = base + pp;
      float xv = 0.f, dv = 0.f;
      if (p < npix) {
        int bb = (int)(p / ((long long)H * W));
        int rem = (int)(p % ((long long)H * W));
        int yy = rem / W, xx = rem % W;
        int sy = wrapi(yy + dy, H), sx = wrapi(xx + dx, W);
        if (c < cin) xv = __bfloat162float(x[(((size_t)bb * H + sy) * W + sx) * cin_p + c]);
        if (c < cout) dv = dz[(size_t)p * cout_p + c];
      }
      xs[pp][c] = xv;
      ds[pp][c] = dv;
    }
    __syncthreads();
    if (ci < cin)
      for (int pp = 0; pp < 64; ++pp) {
        float xv = xs[pp][ci];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fmaf(xv, ds[pp][co0 + q], acc[q]);
      }
    if (tap == 4 && tid < cout)
      for (int pp = 0; pp < 64; ++pp) dbacc += ds[pp][tid];
  }
  if (ci < cin)
    for (int q = 0; q < 4; ++q)
      if (co0 + q < cout) part[(((size_t)chunk * 9 + tap) * kMaxCin + ci) * kMaxCout + co0 + q] = acc[q];
  if (tap == 4 && tid < cout) dbpart[(size_t)chunk * kMaxCout + tid] = dbacc;
}

// Weight gradient of the 32-channel layers on tensor cores (mma.sync m16n8k16, BF16
// operands, FP32 accumulation): the implicit GEMM
//   D[co][tap, ci] = sum_p dz[p][co] x[p + off(tap)][ci],  M = 32 (co), N = 9 x 32, K = pixels.
// A CTA takes a segment of kWgTX pixels of kWgRows consecutive image rows; it keeps the
// three input rows a tap reaches in a ring of shared-memory rows (periodic halo pixels
// included) and the dz row, converted to BF16, beside them; warp w computes tap w's
// 32 x 32 block for all of the CTA's pixels.  Both operands are read with
// ldmatrix.trans from pixel-major rows (a tap's pixel shift is a row offset).  The
// shared-memory pixel stride of 80 bytes makes the eight 16-byte rows of an ldmatrix
// fall in distinct banks.  Pixels past the image edge carry dz = 0.  The bias gradient
// sums the FP32 dz in a fixed order per thread, then over threads in index order.  The
// CTA's partial sums go to part[chunk] like the CUDA-core kernel's, and the same
// reduction adds them in chunk order.
constexpr int kWgTX = 64, kWgRows = 16, kWgS = 40, kWgThreads = 288;

__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const __nv_bfloat16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__global__ void __launch_bounds__(kWgThreads) k_wgrad_mma(const __nv_bfloat16* __restrict__ x, const float* __restrict__ dz,
                                                          int B, int H, int W, int cout, float* __restrict__ part,
                                                          float* __restrict__ dbpart) {
  __shared__ __align__(16) __nv_bfloat16 xs[3][kWgTX + 2][kWgS];
  __shared__ __align__(16) __nv_bfloat16 ds[kWgTX][kWgS];
  __shared__ float dbs[kWgThreads][4];
  const int strips = (W + kWgTX - 1) / kWgTX, rch = (H + kWgRows - 1) / kWgRows;
  const int chunk = blockIdx.x;
  const int b = chunk / (strips * rch), rem = chunk - b * strips * rch;
  const int y0 = (rem / strips) * kWgRows, x0 = (rem % strips) * kWgTX;
  const int y1 = min(H, y0 + kWgRows);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int dy = warp / 3 - 1, dx = warp % 3 - 1;
  float acc[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
  float db4[4] = {0.f, 0.f, 0.f, 0.f};
  // input row yy (periodic) into ring slot `slot`: pixels x0-1 .. x0+kWgTX, 4 x 16 bytes each
  auto stage_x = [&](int yy, int slot) {
    const size_t rowbase = ((size_t)b * H + wrapi(yy, H)) * W;
    for (int t = tid; t < (kWgTX + 2) * 4; t += kWgThreads) {
      const int px = t >> 2, c = (t & 3) * 8;
      const uint4 v = *reinterpret_cast<const uint4*>(x + (rowbase + wrapi(x0 - 1 + px, W)) * 32 + c);
      *reinterpret_cast<uint4*>(&xs[slot][px][c]) = v;
    }
  };
  stage_x(y0 - 1, 0);
  stage_x(y0, 1);
  for (int y = y0; y < y1; ++y) {
    stage_x(y + 1, (y - y0 + 2) % 3);
    {   // dz row y as BF16; thread tid always holds channels (tid & 7) * 4 .. +3
      const size_t rowbase = ((size_t)b * H + y) * W;
      for (int t = tid; t < kWgTX * 8; t += kWgThreads) {
        const int px = t >> 3, c = (t & 7) * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (x0 + px < W) v = *reinterpret_cast<const float4*>(dz + (rowbase + x0 + px) * 32 + c);
        db4[0] += v.x;
        db4[1] += v.y;
        db4[2] += v.z;
        db4[3] += v.w;
        __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
        uint2 pk;
        pk.x = *reinterpret_cast<unsigned*>(&lo);
        pk.y = *reinterpret_cast<unsigned*>(&hi);
        *reinterpret_cast<uint2*>(&ds[px][c]) = pk;
      }
    }
    __syncthreads();
    const int slot = (y + dy - y0 + 1) % 3;
    const int j = lane >> 3, r = lane & 7;
#pragma unroll
    for (int k0 = 0; k0 < kWgTX; k0 += 16) {
      unsigned a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) ldsm_x4_t(a[mt], &ds[k0 + r + 8 * (j >> 1)][mt * 16 + 8 * (j & 1)]);
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        unsigned bq[4];
        ldsm_x4_t(bq, &xs[slot][k0 + r + 8 * (j & 1) + dx + 1][np * 16 + 8 * (j >> 1)]);
        const unsigned b0[2] = {bq[0], bq[1]}, b1[2] = {bq[2], bq[3]};
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma_bf16_16816(acc[mt][2 * np], a[mt], b0);
          mma_bf16_16816(acc[mt][2 * np + 1], a[mt], b1);
        }
      }
    }
    __syncthreads();
  }
  // D[co][ci] of tap `warp`: element e of tile (mt, nt) is co = 16 mt + g (+8 for e >= 2),
  // ci = 8 nt + 2 t (+1 for odd e), g = lane / 4, t = lane % 4
  const int g = lane >> 2, t4 = lane & 3;
  float* pt = part + ((size_t)chunk * 9 + warp) * kMaxCin * kMaxCout;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int co = 16 * mt + g + 8 * (e >> 1), ci = 8 * nt + 2 * t4 + (e & 1);
        if (co < cout) pt[ci * kMaxCout + co] = acc[mt][nt][e];
      }
  dbs[tid][0] = db4[0];
  dbs[tid][1] = db4[1];
  dbs[tid][2] = db4[2];
  dbs[tid][3] = db4[3];
  __syncthreads();
  if (tid < cout) {
    float sdb = 0.f;
    for (int q = tid >> 2; q < kWgThreads; q += 8) sdb += dbs[q][tid & 3];
    dbpart[(size_t)chunk * kMaxCout + tid] = sdb;
  }
}

// dW[tap][ci][co] = sum over chunks in chunk order (deterministic); db likewise.
__global__ void k_wgrad_reduce(const float* __restrict__ part, const float* __restrict__ dbpart, int nchunk, int cin,
                               int cout, float* __restrict__ dw, float* __restrict__ db) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int total = 9 * cin * cout;
  if (t < total) {
    int tap = t / (cin * cout), rem = t % (cin * cout), ci = rem / cout, co = rem % cout;
    float s = 0.f;
    for (int c = 0; c < nchunk; ++c) s += part[(((size_t)c * 9 + tap) * kMaxCin + ci) * kMaxCout + co];
    dw[t] = s;
  } else if (t < total + cout) {
    int co = t - total;
    float s = 0.f;
    for (int c = 0; c < nchunk; ++c) s += dbpart[(size_t)c * kMaxCout + co];
    db[co] = s;
  }
}

// Kernel-layout bf16 weights from the fp32 master [tap][ci][co].
// forward: Wk[co][tap*cin_p + ci]; data gradient (flipped taps, transposed channels):
// Wk[ci][tap'*cout_p + co] with tap' = 8 - tap.
__global__ void k_pack_weights(const float* __restrict__ w, int cin, int cout, int cin_p, int cout_p, int kpad,
                               int transposed, __nv_bfloat16* __restrict__ wk) {
  int rows = transposed ? cin_p : cout_p;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * kpad) return;
  int r = t / kpad, k = t % kpad;
  float v = 0.f;
  if (!transposed) {
    int co = r, tap = k / cin_p, ci = k % cin_p;
    if (k < 9 * cin_p && co < cout && ci < cin) v = w[((size_t)tap * cin + ci) * cout + co];
  } else {
    int ci = r, tapf = k / cout_p, co = k % cout_p;
    if (k < 9 * cout_p && ci < cin && co < cout) v = w[((size_t)(8 - tapf) * cin + ci) * cout + co];
  }
  wk[t] = __float2bfloat16_rn(v);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// MSE over n predictions (channel 0 of an fp32 NHWC tensor with stride cs):
// dy = 2 (yhat - y) / n (bf16 and fp32 copies), loss partials per block.
__global__ void k_mse(const float* __restrict__ yhat, int cs, const float* __restrict__ y, long long n,
                      float* __restrict__ dyf, __nv_bfloat16* __restrict__ dyb, int dcs, float* __restrict__ lpart) {
  __shared__ float red[256];
  float acc = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float d = yhat[i * cs] - y[i];
    acc += d * d;
    float gd = 2.f * d / (float)n;
    for (int c = 0; c < dcs; ++c) {
      dyf[i * dcs + c] = c == 0 ? gd : 0.f;
      dyb[i * dcs + c] = __float2bfloat16_rn(c == 0 ? gd : 0.f);
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
}

size_t conv_smem(int cin_p, int cout_p, int kpad) {
  size_t xs = (size_t)(kTH + 2) * (kTW + 2) * (cin_p / 2 + 4) * 2;
  xs = (xs + 7) & ~(size_t)7;
  return sizeof(__nv_bfloat16) * (xs + (size_t)cout_p * (kpad + 8));
}

int launch_conv(const ConvArgs& A, cudaStream_t s) {
  if (mpfc_cnn_tc_eligible(A.cin_p, A.cout_p, A.W, A.mode))
    return mpfc_cnn_conv_tc(A.x, A.B, A.H, A.W, A.wk, A.bias, A.cout, A.cout_p, A.mode, A.y_bf16, A.y_f32, A.z_f32,
                            A.phi0, A.scale, s);
  long long ntiles = (long long)((A.W + kTW - 1) / kTW) * ((A.H + kTH - 1) / kTH) * A.B;
  const long long cap = 6LL * mpfc::sm_count();
  int grid = (int)(ntiles < cap ? ntiles : cap);
  size_t sm = conv_smem(A.cin_p, A.cout_p, A.kpad);
  if (sm > 48 * 1024) {
    static bool raised = false;
    if (!raised) {
      cudaFuncSetAttribute(k_conv3x3, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
      raised = true;
    }
  }
  k_conv3x3<<<grid, 128, sm, s>>>(A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "k_conv3x3", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  return MPFC_OK;
}

bool cp_ok(int c) { return c == 4 || c == 8 || c == 16 || c == 32; }

}  // namespace

// Per-sample mean of phi^k in two deterministic passes: kMeanBlocks partial sums per
// sample (fixed tree), then one warp per sample adds them in block order.
constexpr int kMeanBlocks = 128;
__global__ void k_mean_partial(const double* __restrict__ phik, long long G, double* __restrict__ part) {
  __shared__ double red[256];
  const int b = blockIdx.y;
  const double* f = phik + (size_t)b * G;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < G; i += (long long)gridDim.x * blockDim.x)
    acc += f[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)b * kMeanBlocks + blockIdx.x] = red[0];
}

__global__ void k_mean_final(const double* __restrict__ part, long long G, double* __restrict__ means) {
  const int b = blockIdx.x, lane = threadIdx.x;
  double s = 0.0;
  for (int i = lane; i < kMeanBlocks; i += 32) s += part[(size_t)b * kMeanBlocks + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) means[b] = s / (double)G;
}

// Network input (4 channels, bf16) from the last three fields, and (optionally) the
// training target, all scaled by the model's normalisation:
//   x0 = (phi^k - mean)/s0, x1 = (phi^k - phi^{k-1})/s1, x2 = (phi^k - 2 phi^{k-1} + phi^{k-2})/s2, x3 = 0,
//   y  = (phi^{k+1} - 2 phi^k + phi^{k-1})/sy   (the error of the linear extrapolation).
__global__ void k_features(const double* __restrict__ p0, const double* __restrict__ p1, const double* __restrict__ p2,
                           const double* __restrict__ pn, long long G, const float* __restrict__ norms,
                           const double* __restrict__ means, __nv_bfloat16* __restrict__ x, float* __restrict__ y) {
  const int b = blockIdx.y;   // sample
  const double inv0 = 1.0 / (double)norms[0], inv1 = 1.0 / (double)norms[1], inv2 = 1.0 / (double)norms[2];
  const double inv3 = 1.0 / (double)norms[3], mean = means[b];
  const size_t off = (size_t)b * G;
  uint2* xo = reinterpret_cast<uint2*>(x) + off;   // 4 bf16 channels = 8 bytes per pixel
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < G; i += (long long)gridDim.x * blockDim.x) {
    const double a = p0[off + i], c1 = p1[off + i], c2 = p2[off + i];
    __nv_bfloat162 lo = __floats2bfloat162_rn((float)((a - mean) * inv0), (float)((a - c1) * inv1));
    __nv_bfloat162 hi = __floats2bfloat162_rn((float)(((a - c1) - (c1 - c2)) * inv2), 0.f);
    xo[i] = make_uint2(*reinterpret_cast<unsigned*>(&lo), *reinterpret_cast<unsigned*>(&hi));
    if (y && pn) y[off + i] = (float)((pn[off + i] - 2.0 * a + c1) * inv3);
  }
}

// Mean of one field into means[0] (partials in means[1 ..]), for the solver's guess.
void mpfc_cnn_mean(const double* phik, long long G, double* means, cudaStream_t s) {
  k_mean_partial<<<dim3(kMeanBlocks, 1), 256, 0, s>>>(phik, G, means + 1);
  k_mean_final<<<1, 32, 0, s>>>(means + 1, G, means);
}

// ---------------------------------------------------------------------------
// C ABI (include/mpfc_cnn.h)
// ---------------------------------------------------------------------------
extern "C" int mpfc_cnn_features(const double* phik, const double* phikm1, const double* phikm2,
                                 const double* phikp1, int B, int H, int W, const float* norms, double* means,
                                 void* x_bf16, float* y_f32, void* stream) {
  if (!phik || !phikm1 || !phikm2 || !norms || !means || !x_bf16 || B < 1 || H < 1 || W < 1) return MPFC_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  long long G = (long long)H * W;
  double* part = means + B;
  k_mean_partial<<<dim3(kMeanBlocks, B), 256, 0, s>>>(phik, G, part);
  k_mean_final<<<B, 32, 0, s>>>(part, G, means);
  const long long per = (G + 255) / 256, cap = (16LL * mpfc::sm_count() + B - 1) / B;
  const dim3 grid((unsigned)(per < cap ? per : cap), (unsigned)B);
  k_features<<<grid, 256, 0, s>>>(phik, phikm1, phikm2, phikp1, G, norms, means, (__nv_bfloat16*)x_bf16, y_f32);
  return cudaGetLastError() == cudaSuccess ? MPFC_OK : MPFC_ERR_CUDA;
}

extern "C" int mpfc_cnn_pack_weights(const float* w, int cin, int cout, int cin_p, int cout_p, int transposed,
                                     void* wk, void* stream) {
  if (!w || !wk || cin < 1 || cout < 1 || cin > cin_p || cout > cout_p) return MPFC_ERR_INVALID;
  if (!transposed && (!cp_ok(cin_p) || (cout_p % 8) || cout_p > kMaxCout)) return MPFC_ERR_INVALID;
  if (transposed && (!cp_ok(cout_p) || (cin_p % 8) || cin_p > kMaxCout)) return MPFC_ERR_INVALID;
  int kin = transposed ? cout_p : cin_p;
  int kpad = (9 * kin + 15) / 16 * 16;
  int rows = transposed ? cin_p : cout_p;
  int n = rows * kpad;
  k_pack_weights<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, cin, cout, cin_p, cout_p, kpad, transposed,
                                                                    (__nv_bfloat16*)wk);
  return cudaGetLastError() == cudaSuccess ? MPFC_OK : MPFC_ERR_CUDA;
}

extern "C" int mpfc_cnn_conv_forward(const void* x, int B, int H, int W, int cin_p, const void* wk, const float* bias,
                                     int cout, int cout_p, int mode, void* y_bf16, float* y_f32, float* z_f32,
                                     void* stream) {
  if (!x || !wk || B < 1 || H < 1 || W < 1 || !cp_ok(cin_p) || cout < 1 || cout > cout_p || cout_p > kMaxCout ||
      (cout_p % 8) || mode < kEpiGeluBf16 || mode > kEpiLinearF32)
    return MPFC_ERR_INVALID;
  if (mode == kEpiGeluBf16 && !y_bf16) return MPFC_ERR_INVALID;
  if (mode == kEpiLinearF32 && !y_f32) return MPFC_ERR_INVALID;
  ConvArgs A{};
  A.x = (const __nv_bfloat16*)x;
  A.wk = (const __nv_bfloat16*)wk;
  A.bias = bias;
  A.B = B;
  A.H = H;
  A.W = W;
  A.cin_p = cin_p;
  A.cout = cout;
  A.cout_p = cout_p;
  A.kpad = (9 * cin_p + 15) / 16 * 16;
  A.mode = mode;
  A.y_bf16 = (__nv_bfloat16*)y_bf16;
  A.y_f32 = y_f32;
  A.z_f32 = z_f32;
  return launch_conv(A, (cudaStream_t)stream);
}

extern "C" int mpfc_cnn_conv_backward_data(const void* dz, int B, int H, int W, int cout_p, const void* wk_t, int cin,
                                           int cin_p, const float* z_prev, void* dzprev_bf16, float* dzprev_f32,
                                           void* stream) {
  if (!dz || !wk_t || !z_prev || !dzprev_bf16 || !dzprev_f32 || !cp_ok(cout_p) || cin < 1 || cin > cin_p ||
      (cin_p % 8) || cin_p > kMaxCout)
    return MPFC_ERR_INVALID;
  ConvArgs A{};
  A.x = (const __nv_bfloat16*)dz;
  A.wk = (const __nv_bfloat16*)wk_t;
  A.bias = nullptr;
  A.B = B;
  A.H = H;
  A.W = W;
  A.cin_p = cout_p;
  A.cout = cin;
  A.cout_p = cin_p;
  A.kpad = (9 * cout_p + 15) / 16 * 16;
  A.mode = kEpiGeluGradBf16;
  A.y_bf16 = (__nv_bfloat16*)dzprev_bf16;
  A.y_f32 = dzprev_f32;
  A.z_f32 = const_cast<float*>(z_prev);
  return launch_conv(A, (cudaStream_t)stream);
}

// Partial-sum slots of the two weight-gradient kernels for a B x H x W batch.
long long wgrad_chunks_scalar(int B, int H, int W) {
  const long long npix = (long long)B * H * W;
  return (npix + kWgChunk - 1) / kWgChunk;
}
long long wgrad_chunks_mma(int B, int H, int W) {
  return (long long)B * ((H + kWgRows - 1) / kWgRows) * ((W + kWgTX - 1) / kWgTX);
}

extern "C" size_t mpfc_cnn_wgrad_scratch_bytes(int B, int H, int W) {
  const long long a = wgrad_chunks_scalar(B, H, W), b = wgrad_chunks_mma(B, H, W);
  const long long nchunk = a > b ? a : b;
  return (size_t)nchunk * (9 * kMaxCin * kMaxCout + kMaxCout) * sizeof(float);
}

extern "C" int mpfc_cnn_conv_backward_weight(const void* x, int B, int H, int W, int cin, int cin_p, const float* dz,
                                             int cout, int cout_p, float* dw, float* db, void* scratch,
                                             void* stream) {
  if (!x || !dz || !dw || !db || !scratch || cin < 1 || cin > cin_p || cin > kMaxCin || cout < 1 ||
      cout > cout_p || cout > kMaxCout || !cp_ok(cin_p))
    return MPFC_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  float* part = (float*)scratch;
  int nchunk;
  if (cin == 32 && cin_p == 32 && cout_p == 32) {
    // the 32 -> 32 layers: tensor cores
    nchunk = (int)wgrad_chunks_mma(B, H, W);
    float* dbpart = part + (size_t)nchunk * 9 * kMaxCin * kMaxCout;
    k_wgrad_mma<<<nchunk, kWgThreads, 0, s>>>((const __nv_bfloat16*)x, dz, B, H, W, cout, part, dbpart);
    const int total = 9 * cin * cout + cout;
    k_wgrad_reduce<<<(total + 255) / 256, 256, 0, s>>>(part, dbpart, nchunk, cin, cout, dw, db);
    return cudaGetLastError() == cudaSuccess ? MPFC_OK : MPFC_ERR_CUDA;
  }
  // layers with 4-channel inputs or 1-channel outputs: CUDA cores, FP32 dz
  nchunk = (int)wgrad_chunks_scalar(B, H, W);
  float* dbpart = part + (size_t)nchunk * 9 * kMaxCin * kMaxCout;
  k_wgrad_partial<<<dim3(nchunk, 9), 256, 0, s>>>((const __nv_bfloat16*)x, dz, B, H, W, cin_p, cin, cout_p, cout,
                                                 part, dbpart);
  int total = 9 * cin * cout + cout;
  k_wgrad_reduce<<<(total + 255) / 256, 256, 0, s>>>(part, dbpart, nchunk, cin, cout, dw, db);
  return cudaGetLastError() == cudaSuccess ? MPFC_OK : MPFC_ERR_CUDA;
}

extern "C" int mpfc_cnn_mse(const float* yhat, int yhat_stride, const float* y, long long n, float* dy_f32,
                            void* dy_bf16, int dy_stride, float* loss_partials, int nblocks, void* stream) {
  if (!yhat || !y || !dy_f32 || !dy_bf16 || !loss_partials || n < 1 || nblocks < 1 || nblocks > 4096)
    return MPFC_ERR_INVALID;
  k_mse<<<nblocks, 256, 0, (cudaStream_t)stream>>>(yhat, yhat_stride, y, n, dy_f32, (__nv_bfloat16*)dy_bf16,
                                                   dy_stride, loss_partials);
  return cudaGetLastError() == cudaSuccess ? MPFC_OK : MPFC_ERR_CUDA;
}

extern "C" int mpfc_cnn_adam(float* param, const float* grad, float* m, float* v, int n, float lr, float beta1,
                             float beta2, float eps, int t, void* stream) {
  if (!param || !grad || !m || !v || n < 1 || t < 1) return MPFC_ERR_INVALID;
  float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
  k_adam<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(param, grad, m, v, n, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? MPFC_OK : MPFC_ERR_CUDA;
}

// Used by the solver's learned guess (guess_cnn.cu): the last layer adds its output,
// scaled, to the FP64 initial guess.
int mpfc_cnn_conv_guess(const void* x, int H, int W, int cin_p, const void* wk, const float* bias, double* phi0,
                        double scale, cudaStream_t s) {
  ConvArgs A{};
  A.x = (const __nv_bfloat16*)x;
  A.wk = (const __nv_bfloat16*)wk;
  A.bias = bias;
  A.B = 1;
  A.H = H;
  A.W = W;
  A.cin_p = cin_p;
  A.cout = 1;
  A.cout_p = 8;
  A.kpad = (9 * cin_p + 15) / 16 * 16;
  A.mode = kEpiGuess;
  A.phi0 = phi0;
  A.scale = scale;
  return launch_conv(A, s);
}

int mpfc_cnn_conv_layer(const void* x, int H, int W, int cin_p, const void* wk, const float* bias, int cout,
                        void* y_bf16, cudaStream_t s) {
  ConvArgs A{};
  A.x = (const __nv_bfloat16*)x;
  A.wk = (const __nv_bfloat16*)wk;
  A.bias = bias;
  A.B = 1;
  A.H = H;
  A.W = W;
  A.cin_p = cin_p;
  A.cout = cout;
  A.cout_p = 32;
  A.kpad = (9 * cin_p + 15) / 16 * 16;
  A.mode = kEpiGeluBf16;
  A.y_bf16 = (__nv_bfloat16*)y_bf16;
  return launch_conv(A, s);
}
