// Learned heuristic network: crop extraction, BF16 forward and backward
// passes on the tensor cores, and Adam (training and inference kernels).
//
// The paper's multi-heuristic search (Sec. IV-B/C) admits any inadmissible
// heuristic and names learned ones as the next step (Sec. IV-C, Sec. VI); it
// fixes no network. This one predicts y = log(1 + edge cost) of one MSGT
// successor from a 2 x 64 x 64 crop (observed depth, parent z-buffer) centred
// on the projected hypothesis, and a one-hot of (mesh, yaw):
//   conv 3x3 2->32 s1, 32->64 s2, 64->128 s2, 128->128 s2 (pad 1, ReLU)
//   -> flatten (h, w, c) ++ one-hot -> FC 96 (ReLU) -> FC 1; loss 0.5 (pred - y)^2
//
// Data layout: activations NHWC bfloat16. Every convolution is one GEMM over
// rows = output pixels (N x Ho x Wo) and columns = (tap, channel) (K = 9 Cin,
// padded to 32): the 2-channel input layer through an explicit im2col, the
// others by gathering 16-byte chunks of the NHWC input straight into shared
// memory (implicit im2col, zero padding through the copy's source size). The
// GEMM is mma.sync m16n8k16 (BF16 in, FP32 accumulate) fed by a 3-stage
// cp.async pipeline and ldmatrix (.trans for MN-contiguous operands). Weight
// gradients reduce over pixels with both operands read in place, split along
// the reduction and summed in a fixed order (deterministic). Gradients between
// layers are rounded to bfloat16, like the activations; weights keep an FP32
// master copy updated by Adam and re-rounded to bfloat16 after each step.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "perch_ctx.h"

using namespace perch;
typedef __nv_bfloat16 bf16;

namespace {

constexpr int kCrop = 64;
constexpr int kHidden = 96;
constexpr int kConvs = 4;
constexpr int kCin[kConvs] = {2, 32, 64, 128};
constexpr int kCout[kConvs] = {32, 64, 128, 128};
constexpr int kStride[kConvs] = {1, 2, 2, 2};
constexpr int kHin[kConvs] = {64, 64, 32, 16};  // input side of each layer
constexpr int kFeat = 128 * 8 * 8;               // flattened last conv output
constexpr float kMissing = -4.0f, kClamp = 3.0f;
constexpr double kScale = 10.0;  // per metre

int round32(int v) { return (v + 31) / 32 * 32; }
int kp_of(int l) { return round32(9 * kCin[l]); }

// ---------------------------------------------------------------- GEMM
constexpr int BM = 128, BK = 32, LDS = BK + 8, STAGES = 3;
enum { EPI_BIAS_RELU = 0, EPI_F32 = 1, EPI_BF16 = 2, EPI_DGRAD = 3 };

struct GemmArgs {
  const bf16* A;  // [M][lda], K-contiguous
  long long lda;
  const bf16* B;  // [N][ldb], K-contiguous
  long long ldb;
  int M, N, K, Ksplit;  // split z covers columns [z Ksplit, min(K, (z + 1) Ksplit))
  float* Cf;            // EPI_F32 output (partial z at Cf + z split_stride)
  bf16* Cb;             // EPI_BIAS_RELU output
  long long ldc;
  int grp;              // output row m lives at (m / grp) ldg + (m % grp) ldc
  long long ldg;
  long long split_stride;
  const float* bias;
  // implicit im2col (CONV = 1: A, CONV = 2: B): the operand is the NHWC
  // input of a 3x3 pad-1 convolution with power-of-two channels and output
  // side; pixel index (n, i, j) and column index (tap, c), tap = 3 kh + kw
  int cH, cs, lg_c, lg_wo;
  // fused data gradient of a stride-2 convolution (CONV = 3, EPI_DGRAD), one
  // parity class (par_h, par_w) of the input pixels: rows = the class's
  // pixels (n, a, b) at (2a + par_h, 2b + par_w); columns = input channels;
  // K = (tap of the class, output channel). A gathers dz, B reads W in place,
  // the epilogue applies the ReLU mask of the layer input and scatters rows
  // back to NHWC.
  int par_h, par_w, ntw, dg_lg_ho, dg_lg_co, dg_H, dg_cin, dg_kp;
  const bf16* mask;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool pred) {
  const int sz = pred ? 16 : 0;  // src-size 0: the 16 bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(sz));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C[M x N] = A B^T over K. A is K-contiguous (AK: element (m, k) at
// m lda + k) or M-contiguous (element (m, k) at k lda + m); B likewise
// (BKC: (n, k) at n ldb + k, else k ldb + n). MN-contiguous operands are
// staged as [k][m] tiles and fed to the tensor cores with ldmatrix .trans, so
// weight and data gradients need no transposed copies. 256 threads; CTA tile
// 128 x BN; warp tile (128 / (8 / (BN / 32))) x 32. K and Ksplit multiples of
// 32; an MN-contiguous operand needs its M (or N) to be a multiple of 8.
// Source of one 16-byte chunk of an implicit im2col operand: output pixel
// `m`, columns k .. k + 7 (one tap, 8 channels); nullptr where the tap falls
// in the zero padding.
__device__ __forceinline__ const bf16* conv_src(const GemmArgs& p, const bf16* x, int m, int k) {
  const int tap = k >> p.lg_c, c = k & ((1 << p.lg_c) - 1);
  const int wo = 1 << p.lg_wo;
  const int j = m & (wo - 1), i = (m >> p.lg_wo) & (wo - 1), n = m >> (2 * p.lg_wo);
  const int r = p.cs * i - 1 + tap / 3, cc = p.cs * j - 1 + tap % 3;
  if (tap >= 9 || r < 0 || r >= p.cH || cc < 0 || cc >= p.cH) return nullptr;
  return x + ((((long long)n * p.cH + r) * p.cH + cc) << p.lg_c) + c;
}

// Taps of one parity of a stride-2, pad-1, 3x3 convolution's input: an even
// coordinate 2a is read by kernel offset 1 of output a; an odd one 2a + 1 by
// offset 0 of output a + 1 and offset 2 of output a.
__device__ __forceinline__ void dg_tap(int par, int t, int& kofs, int& d) {
  kofs = par == 0 ? 1 : (t == 0 ? 0 : 2);
  d = (par == 1 && t == 0) ? 1 : 0;
}

// A chunk of the fused data gradient: class pixel m, columns k .. k + 7 (one
// tap, 8 output channels) of dz; nullptr where that output pixel is outside.
__device__ __forceinline__ const bf16* dgrad_a_src(const GemmArgs& p, int m, int k) {
  const int t = k >> p.dg_lg_co, o = k & ((1 << p.dg_lg_co) - 1);
  int kh, dh, kw, dw;
  dg_tap(p.par_h, t / p.ntw, kh, dh);
  dg_tap(p.par_w, t % p.ntw, kw, dw);
  const int ho = 1 << p.dg_lg_ho;
  const int b = m & (ho - 1), a = (m >> p.dg_lg_ho) & (ho - 1), n = m >> (2 * p.dg_lg_ho);
  const int i = a + dh, j = b + dw;
  if (i >= ho || j >= ho) return nullptr;
  return p.A + ((((long long)n * ho + i) * ho + j) << p.dg_lg_co) + o;
}

// B chunk: K row (tap, o), input channels n .. n + 7 of W[o][kh][kw][.]
__device__ __forceinline__ const bf16* dgrad_b_src(const GemmArgs& p, int k, int n) {
  const int t = k >> p.dg_lg_co, o = k & ((1 << p.dg_lg_co) - 1);
  int kh, dh, kw, dw;
  dg_tap(p.par_h, t / p.ntw, kh, dh);
  dg_tap(p.par_w, t % p.ntw, kw, dw);
  return p.B + (long long)o * p.dg_kp + (kh * 3 + kw) * p.dg_cin + n;
}

template <int BN, int EPI, bool AK, bool BKC, int CONV>
__global__ void __launch_bounds__(256) k_gemm(GemmArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int A_LD = AK ? LDS : BM + 8, A_STAGE = AK ? BM * LDS : BK * (BM + 8);
  constexpr int B_LD = BKC ? LDS : BN + 8, B_STAGE = BKC ? BN * LDS : BK * (BN + 8);
  bf16* As = reinterpret_cast<bf16*>(smem_raw);  // [STAGES][A_STAGE]
  bf16* Bs = As + STAGES * A_STAGE;               // [STAGES][B_STAGE]
  constexpr int WN = BN / 32, WM = 8 / WN, TM = BM / WM, MI = TM / 16;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp / WN, wn = warp % WN;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * p.Ksplit;
  const int kend = min(p.K, kbeg + p.Ksplit);
  const int KT = kend > kbeg ? (kend - kbeg) / BK : 0;
  float acc[MI][4][4];
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;

  auto load = [&](int stage, int kt) {
    const int k0 = kbeg + kt * BK;
    bf16* as = As + stage * A_STAGE;
    bf16* bs = Bs + stage * B_STAGE;
    if (AK) {
      for (int c = tid; c < BM * 4; c += 256) {
        const int r = c >> 2, q = c & 3, gm = m0 + r;
        bool ok = gm < p.M;
        const bf16* src = p.A;
        if (CONV == 1 || CONV == 3) {
          const bf16* g = ok ? (CONV == 1 ? conv_src(p, p.A, gm, k0 + q * 8) : dgrad_a_src(p, gm, k0 + q * 8))
                             : nullptr;
          ok = g != nullptr;
          if (ok) src = g;
        } else if (ok) {
          src = p.A + (long long)gm * p.lda + k0 + q * 8;
        }
        cp_async16(smem_addr(as + r * A_LD + q * 8), src, ok);
      }
    } else {
      for (int c = tid; c < BK * (BM / 8); c += 256) {
        const int r = c / (BM / 8), q = c % (BM / 8), gm = m0 + q * 8;
        const bool ok = gm < p.M;
        const bf16* src = ok ? p.A + (long long)(k0 + r) * p.lda + gm : p.A;
        cp_async16(smem_addr(as + r * A_LD + q * 8), src, ok);
      }
    }
    if (BKC) {
      for (int c = tid; c < BN * 4; c += 256) {
        const int r = c >> 2, q = c & 3, gn = n0 + r;
        const bool ok = gn < p.N;
        const bf16* src = ok ? p.B + (long long)gn * p.ldb + k0 + q * 8 : p.B;
        cp_async16(smem_addr(bs + r * B_LD + q * 8), src, ok);
      }
    } else {
      for (int c = tid; c < BK * (BN / 8); c += 256) {
        const int r = c / (BN / 8), q = c % (BN / 8), gn = n0 + q * 8;
        bool ok = gn < p.N;
        const bf16* src = p.B;
        if (CONV == 2) {
          const bf16* g = ok ? conv_src(p, p.B, k0 + r, gn) : nullptr;
          ok = g != nullptr;
          if (ok) src = g;
        } else if (CONV == 3) {
          if (ok) src = dgrad_b_src(p, k0 + r, gn);
        } else if (ok) {
          src = p.B + (long long)(k0 + r) * p.ldb + gn;
        }
        cp_async16(smem_addr(bs + r * B_LD + q * 8), src, ok);
      }
    }
  };
#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < KT) load(s, s);
    cp_commit();
  }
  for (int kt = 0; kt < KT; ++kt) {
    cp_wait<STAGES - 2>();
    __syncthreads();  // stage kt landed for every thread; stage kt - 1 is free
    {
      const int nk = kt + STAGES - 1;
      if (nk < KT) load(nk % STAGES, nk);
      cp_commit();
    }
    const bf16* as = As + (kt % STAGES) * A_STAGE;
    const bf16* bs = Bs + (kt % STAGES) * B_STAGE;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      uint32_t af[MI][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < MI; ++i) {
        const int mb = wm * TM + i * 16;
        if (AK) {
          const int row = mb + (lane & 15), col = kk * 16 + (lane >> 4) * 8;
          ldsm_x4(smem_addr(as + row * A_LD + col), af[i][0], af[i][1], af[i][2], af[i][3]);
        } else {  // matrices (m, k) blocks: (0, 0), (8, 0), (0, 8), (8, 8)
          const int q = lane >> 3;
          const int mm = mb + 8 * (q & 1), kr = kk * 16 + 8 * (q >> 1) + (lane & 7);
          ldsm_x4_t(smem_addr(as + kr * A_LD + mm), af[i][0], af[i][1], af[i][2], af[i][3]);
        }
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int nb = wn * 32 + j * 16;
        if (BKC) {
          const int row = nb + (lane & 7) + ((lane >> 4) << 3);
          const int col = kk * 16 + ((lane >> 3) & 1) * 8;
          ldsm_x4(smem_addr(bs + row * B_LD + col), bfr[2 * j][0], bfr[2 * j][1], bfr[2 * j + 1][0],
                  bfr[2 * j + 1][1]);
        } else {  // matrices (n, k) blocks: (0, 0), (0, 8), (8, 0), (8, 8)
          const int q = lane >> 3;
          const int nn = nb + 8 * (q >> 1), kr = kk * 16 + 8 * (q & 1) + (lane & 7);
          ldsm_x4_t(smem_addr(bs + kr * B_LD + nn), bfr[2 * j][0], bfr[2 * j][1], bfr[2 * j + 1][0],
                    bfr[2 * j + 1][1]);
        }
      }
#pragma unroll
      for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j][0], bfr[j][1]);
    }
  }
  cp_wait<0>();
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = m0 + wm * TM + i * 16 + g + h * 8;
        const int col = n0 + wn * 32 + j * 8 + 2 * t;
        if (row >= p.M || col >= p.N) continue;
        float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
        if (EPI == EPI_DGRAD) {  // class pixel -> NHWC input pixel, times the ReLU mask
          const int ho = 1 << p.dg_lg_ho;
          const int b = row & (ho - 1), a = (row >> p.dg_lg_ho) & (ho - 1), n = row >> (2 * p.dg_lg_ho);
          const long long o =
              (((long long)n * p.dg_H + 2 * a + p.par_h) * p.dg_H + 2 * b + p.par_w) * p.dg_cin + col;
          const __nv_bfloat162 x = *reinterpret_cast<const __nv_bfloat162*>(p.mask + o);
          if (!(__low2float(x) > 0.0f)) v0 = 0.0f;
          if (!(__high2float(x) > 0.0f)) v1 = 0.0f;
          *reinterpret_cast<__nv_bfloat162*>(p.Cb + o) = __floats2bfloat162_rn(v0, v1);
          continue;
        }
        const long long off = (long long)(row / p.grp) * p.ldg + (long long)(row % p.grp) * p.ldc + col;
        if (EPI == EPI_BIAS_RELU) {
          v0 = fmaxf(v0 + p.bias[col], 0.0f);
          v1 = fmaxf(v1 + p.bias[col + 1], 0.0f);
          *reinterpret_cast<__nv_bfloat162*>(p.Cb + off) = __floats2bfloat162_rn(v0, v1);
        } else if (EPI == EPI_BF16) {
          *reinterpret_cast<__nv_bfloat162*>(p.Cb + off) = __floats2bfloat162_rn(v0, v1);
        } else {
          *reinterpret_cast<float2*>(p.Cf + (long long)blockIdx.z * p.split_stride + off) = make_float2(v0, v1);
        }
      }
}

template <int BN, int EPI, bool AK, bool BKC, int CONV>
cudaError_t gemm_bn(const GemmArgs& p, int splits, cudaStream_t s) {
  constexpr int A_STAGE = AK ? BM * LDS : BK * (BM + 8), B_STAGE = BKC ? BN * LDS : BK * (BN + 8);
  const int smem = STAGES * (A_STAGE + B_STAGE) * (int)sizeof(bf16);
  cudaError_t e =
      cudaFuncSetAttribute(k_gemm<BN, EPI, AK, BKC, CONV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((p.N + BN - 1) / BN, (p.M + BM - 1) / BM, splits);
  k_gemm<BN, EPI, AK, BKC, CONV><<<grid, 256, smem, s>>>(p);
  return cudaGetLastError();
}

// C = A B^T (layouts as k_gemm); `splits` CTAs along K, each writing its
// partial at Cf + z split_stride (EPI_F32) or, with one split, the epilogue.
template <int EPI, bool AK = true, bool BKC = true, int CONV = 0>
cudaError_t gemm(GemmArgs p, int splits, cudaStream_t s) {
  if (p.grp <= 0) {
    p.grp = 1 << 30;
    p.ldg = 0;
  }
  if ((!AK && p.M % 8) || (!BKC && p.N % 8) || p.K % 32 || p.Ksplit % 32) return cudaErrorInvalidValue;
  if (CONV && p.lg_c < 3) return cudaErrorInvalidValue;  // chunks of 8 channels within one tap
  if (p.N <= 32) return gemm_bn<32, EPI, AK, BKC, CONV>(p, splits, s);
  if (p.N <= 64) return gemm_bn<64, EPI, AK, BKC, CONV>(p, splits, s);
  return gemm_bn<128, EPI, AK, BKC, CONV>(p, splits, s);
}

// ------------------------------------------------- tcgen05 convolution
// Forward 3x3 convolution with implicit im2col (layers 2-4) on the
// fifth-generation tensor cores: C[M x N] = A B^T, A the im2col rows of the
// NHWC input (conv_src), B the weights [N][K]. One CTA of 256 threads owns a
// 128-row tile and all N (64 or 128) columns; its FP32 accumulator lives in
// tensor memory (N columns, lanes = rows). K advances BK columns per step
// through a ring of S shared-memory stages filled by cp.async in the
// canonical no-swizzle K-major layout: core matrices of 8 rows x 16 bytes,
// the K-adjacent ones 128 bytes apart, the row-adjacent ones BK / 8 x 128
// bytes apart. One thread issues the step's BK / 16 m128 nN k16 MMAs and
// commits them to the stage's mbarrier, which frees the stage for the copy
// of step + S. The epilogue reads the accumulator back with tcgen05.ld (warp
// w: rows 32 (w mod 4) .. + 31, columns of half w / 4), adds the bias,
// applies ReLU and stores bfloat16 rows (GemmArgs addressing). Every wait is
// bounded; a wait that gives up sets *err and skips the stores, and the
// tensor memory is freed all the same.
constexpr int kTcRows = 128, kTcThreads = 256;

template <int BK>
__device__ __forceinline__ uint32_t tc_canon(int r, int kc) {  // (row r, 16-byte chunk kc) in a stage
  return (uint32_t)((r >> 3) * (BK / 8) * 128 + kc * 128 + (r & 7) * 16);
}
// shared-memory matrix descriptor: start address, leading (K) byte offset
// 128, stride (row-group) byte offset, descriptor version 1, no swizzle
template <int BK>
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)((BK / 8) * 128 >> 4) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N
template <int N>
__device__ __forceinline__ uint32_t tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}
__device__ __forceinline__ void tc_mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ uint64_t tc_now() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait for the phase of the given parity: bounded by polls and by 2 s
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = tc_now();
  for (int i = 0; i < (1 << 22); ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 255) == 255 && tc_now() - t0 > 2000000000ull) break;
  }
  return false;
}

template <int N, int BK, int S>
__global__ void __launch_bounds__(kTcThreads) k_conv_tc(GemmArgs p, int* err) {
  static_assert(N == 64 || N == 128, "N must be 64 or 128");
  static_assert(BK % 16 == 0, "BK must be a multiple of 16");
  constexpr int CH = BK / 8, A_BYTES = kTcRows * BK * 2, STAGE = A_BYTES + N * BK * 2;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[S];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTcRows, nk = p.K / BK;
  const uint32_t sbase = smem_addr(smem);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) tc_mbar_init(&bar[s]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // N columns of tensor memory for the accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                 "r"(N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  auto load = [&](int ks) {  // this thread's share of step ks's A and B chunks
    const uint32_t a = sbase + (uint32_t)((ks % S) * STAGE), b = a + A_BYTES;
    const int k0 = ks * BK;
    for (int i = tid; i < kTcRows * CH; i += kTcThreads) {
      const int r = i / CH, kc = i % CH, m = m0 + r;
      const bf16* src = m < p.M ? conv_src(p, p.A, m, k0 + 8 * kc) : nullptr;
      cp_async16(a + tc_canon<BK>(r, kc), src ? src : p.A, src != nullptr);
    }
    for (int i = tid; i < N * CH; i += kTcThreads) {
      const int n = i / CH, kc = i % CH;
      cp_async16(b + tc_canon<BK>(n, kc), p.B + (long long)n * p.ldb + k0 + 8 * kc, true);
    }
  };

  for (int ks = 0; ks < S - 1; ++ks) {
    if (ks < nk) load(ks);
    cp_commit();
  }
  bool ok = true;
  int last = -1;  // last step whose MMAs were issued (the same in every thread)
  for (int ks = 0; ks < nk; ++ks) {
    const int kl = ks + S - 1;  // the step loaded now, into the stage step ks - 1 used
    if (kl < nk) {
      if (kl >= S) ok = ok && tc_wait(&bar[kl % S], (uint32_t)(((kl - S) / S) & 1));
      if (ok) load(kl);
    }
    cp_commit();
    cp_wait<S - 1>();  // this thread's copies of step ks have landed
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
    ok = __syncthreads_and(ok);
    if (ok) last = ks;
    if (ok && tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a = sbase + (uint32_t)((ks % S) * STAGE), b = a + A_BYTES;
      for (int j = 0; j < BK / 16; ++j) {
        const uint64_t ad = tc_desc<BK>(a + 256 * j), bd = tc_desc<BK>(b + 256 * j);
        const uint32_t acc = (ks | j) != 0;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(tc_idesc<N>()), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&bar[ks % S]))
                   : "memory");
    }
  }
  cp_wait<0>();
  // the last commit covers every MMA before it; wait for it (bounded) even
  // after a failure, so that no MMA still writes the tensor memory freed below
  if (last >= 0 && !tc_wait(&bar[last % S], (uint32_t)((last / S) & 1))) ok = false;
  ok = __syncthreads_and(ok && last == nk - 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int q = warp & 3, half = warp >> 2;  // TMEM lanes 32q .. 32q + 31, columns of this half
  const int row = m0 + 32 * q + lane;
  const long long off = (long long)(row / p.grp) * p.ldg + (long long)(row % p.grp) * p.ldc;
  if (ok) {
    for (int c0 = half * (N / 2); c0 < (half + 1) * (N / 2); c0 += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < p.M) {
        uint32_t o[8];
        for (int e = 0; e < 8; ++e) {
          const float x0 = fmaxf(__uint_as_float(v[2 * e]) + p.bias[c0 + 2 * e], 0.0f);
          const float x1 = fmaxf(__uint_as_float(v[2 * e + 1]) + p.bias[c0 + 2 * e + 1], 0.0f);
          const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
          o[e] = *reinterpret_cast<const uint32_t*>(&h);
        }
        uint4* dst = reinterpret_cast<uint4*>(p.Cb + off + c0);
        dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
        dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
      }
    }
  } else if (tid == 0) {
    atomicOr(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(N) : "memory");
}

template <int N, int BK, int S>
cudaError_t conv_tc_t(const GemmArgs& p, int* err, cudaStream_t s) {
  constexpr int smem = S * (kTcRows + N) * BK * 2;
  cudaError_t e = cudaFuncSetAttribute(k_conv_tc<N, BK, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_conv_tc<N, BK, S><<<(unsigned)((p.M + kTcRows - 1) / kTcRows), kTcThreads, smem, s>>>(p, err);
  return cudaGetLastError();
}

// C = relu(A B^T + bias) for one implicit-im2col convolution layer on the
// tcgen05 path (N = 64 or 128, K a multiple of 32, 8-channel chunks). Steps
// of 64 columns where K allows, else 32.
cudaError_t conv_tc(GemmArgs p, int* err, cudaStream_t s) {
  if (p.grp <= 0) {
    p.grp = 1 << 30;
    p.ldg = 0;
  }
  if ((p.N != 64 && p.N != 128) || p.K % 32 || p.lg_c < 3 || p.ldc % 8 || p.ldg % 8) return cudaErrorInvalidValue;
  const bool k64 = p.K % 64 == 0;
  if (p.N == 64) return k64 ? conv_tc_t<64, 64, 4>(p, err, s) : conv_tc_t<64, 32, 4>(p, err, s);
  return k64 ? conv_tc_t<128, 64, 3>(p, err, s) : conv_tc_t<128, 32, 4>(p, err, s);
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

void set_conv(GemmArgs& p, int l) {
  p.cH = kHin[l];
  p.cs = kStride[l];
  p.lg_c = ilog2(kCin[l]);
  p.lg_wo = ilog2(kHin[l] / kStride[l]);
}

// splits along K so that the grid has about two CTAs per SM (each split a
// multiple of 32 long, at least 256)
int choose_splits(int M, int N, int K, int* ksplit) {
  const int bn = N <= 32 ? 32 : N <= 64 ? 64 : 128;
  const int tiles = ((M + BM - 1) / BM) * ((N + bn - 1) / bn);
  int S = std::max(1, std::min((2 * 152 + tiles - 1) / tiles, K / 256));
  int ks = (K / S + 31) / 32 * 32;
  S = (K + ks - 1) / ks;
  *ksplit = ks;
  return S;
}

// ---------------------------------------------------------------- layout kernels
// im2col of the 2-channel input layer (stride 1, Kp = 32): one thread per
// output pixel gathers its 9 taps (4 bytes each) and writes one 64-byte row
__global__ void k_im2col_c2(const uint32_t* __restrict__ x, int N, int H, int W, uint4* __restrict__ col) {
  const long long total = (long long)N * H * W;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < total;
       m += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(m % W), i = (int)((m / W) % H);
    const long long n = m / ((long long)W * H);
    uint32_t v[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = 0u;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int r = i - 1 + tap / 3, c = j - 1 + tap % 3;
      if (r >= 0 && r < H && c >= 0 && c < W) v[tap] = x[(n * H + r) * W + c];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) col[m * 4 + q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  }
}

// part[b][c] = sum of column c over rows [b R, (b + 1) R) of a bfloat16
// [M][C] matrix (bias gradients); 256 threads, 256 / C row groups.
__global__ void k_col_sum(const bf16* __restrict__ in, long long M, int C, int R, float* __restrict__ part) {
  __shared__ float red[256];
  const int G = 256 / C;
  const int c = threadIdx.x % C, grp = threadIdx.x / C;
  const long long r0 = (long long)blockIdx.x * R;
  const long long r1 = min(M, r0 + R);
  float a = 0.0f;
  if (grp < G)
    for (long long r = r0 + grp; r < r1; r += G) a += __bfloat162float(in[r * C + c]);
  red[threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.x < C) {
    float v = 0.0f;
    for (int k = 0; k < G; ++k) v += red[k * C + threadIdx.x];
    part[(long long)blockIdx.x * C + threadIdx.x] = v;
  }
}

// out[r][c] = bf16(relu(sum over z of part[z][r][c] + bias[c])) (split-K FC1)
__global__ void k_splits_bias_relu(const float* __restrict__ part, int splits, long long rows, int C,
                                   const float* __restrict__ bias, bf16* __restrict__ out) {
  const long long n = rows * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    float a = 0.0f;
    for (int z = 0; z < splits; ++z) a += part[(long long)z * n + e];
    out[e] = __float2bfloat16_rn(fmaxf(a + bias[e % C], 0.0f));
  }
}

// out[e] = sum over z of part[z][e] for many partials and few outputs: 32
// outputs per block, blockDim / 32 partial groups per output (at most 32),
// then a fixed-order sum of the groups (deterministic).
__global__ void k_split_sum_wide(const float* __restrict__ part, int splits, long long n, float* __restrict__ out) {
  __shared__ float red[32][33];
  const int G = blockDim.x >> 5;
  const long long e = (long long)blockIdx.x * 32 + (threadIdx.x & 31);
  const int g = threadIdx.x >> 5;
  float a = 0.0f;
  if (e < n)
    for (int z = g; z < splits; z += G) a += part[(long long)z * n + e];
  red[g][threadIdx.x & 31] = a;
  __syncthreads();
  if (threadIdx.x < 32 && e < n) {
    float v = 0.0f;
    for (int k = 0; k < G; ++k) v += red[k][threadIdx.x];
    out[e] = v;
  }
}


// one-hot columns of the FC input: feat[n][kFeat + j] = [j == idx[n]] (ragged rows zero)
__global__ void k_onehot(const int32_t* __restrict__ idx, int n, int n_rows, int n_onehot_pad, long long ldf,
                         bf16* __restrict__ feat) {
  const long long total = (long long)n_rows * n_onehot_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % n_onehot_pad);
    const int r = (int)(e / n_onehot_pad);
    const bool on = r < n && idx[r] == j;
    feat[(long long)r * ldf + kFeat + j] = __float2bfloat16_rn(on ? 1.0f : 0.0f);
  }
}

// pred[n] = h1[n] . bf16(w2) + b2; with a target: err[n] = pred - y
__global__ void k_fc2(const bf16* __restrict__ h1, const float* __restrict__ w2, const float* __restrict__ b2, int n,
                      float* __restrict__ pred, const float* __restrict__ target, float* __restrict__ err) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  float a = 0.0f;
  for (int j = lane; j < kHidden; j += 32)
    a += __bfloat162float(h1[(long long)warp * kHidden + j]) * __bfloat162float(__float2bfloat16_rn(w2[j]));
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) {
    const float pr = a + b2[0];
    if (pred) pred[warp] = pr;
    if (target) err[warp] = pr - target[warp];
  }
}

// loss = mean 0.5 err^2 and the gradient of b2 (one block)
__global__ void k_fc2_loss(const float* __restrict__ err, int n, float* __restrict__ g_b2, float* __restrict__ loss) {
  __shared__ float red[2][32];
  const float inv = 1.0f / (float)n;
  float l = 0.0f, gb = 0.0f;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    l += 0.5f * err[r] * err[r];
    gb += err[r] * inv;
  }
  for (int o = 16; o > 0; o >>= 1) {
    l += __shfl_xor_sync(0xffffffffu, l, o);
    gb += __shfl_xor_sync(0xffffffffu, gb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = l;
    red[1][threadIdx.x >> 5] = gb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.0f, b = 0.0f;
    for (int k = 0; k < (int)blockDim.x / 32; ++k) {
      a += red[0][k];
      b += red[1][k];
    }
    if (loss) *loss = a * inv;
    g_b2[0] = b;
  }
}

// gradient of w2: one block per hidden unit j, sum over the batch
__global__ void k_fc2_wgrad(const bf16* __restrict__ h1, const float* __restrict__ err, int n, float* __restrict__ g_w2) {
  __shared__ float red[32];
  const int j = blockIdx.x;
  const float inv = 1.0f / (float)n;
  float a = 0.0f;
  for (int r = threadIdx.x; r < n; r += blockDim.x) a += err[r] * inv * __bfloat162float(h1[(long long)r * kHidden + j]);
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.0f;
    for (int k = 0; k < (int)blockDim.x / 32; ++k) v += red[k];
    g_w2[j] = v;
  }
}

// dz1 = (err / n) bf16(w2) [h1 > 0]
__global__ void k_fc2_dz1(const bf16* __restrict__ h1, const float* __restrict__ w2, const float* __restrict__ err,
                          int n, bf16* __restrict__ dz1) {
  const float inv = 1.0f / (float)n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * kHidden;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / kHidden), j = (int)(e % kHidden);
    float v = 0.0f;
    if (__bfloat162float(h1[e]) > 0.0f) v = err[r] * inv * __bfloat162float(__float2bfloat16_rn(w2[j]));
    dz1[e] = __float2bfloat16_rn(v);
  }
}

// dz of the last convolution: dfeat (fp32, [n][kFeat]) times [x4 > 0], where
// x4 is read back from the FC input rows
__global__ void k_feat_relu_grad(const float* __restrict__ dfeat, const bf16* __restrict__ feat, long long ldf,
                                 int n, bf16* __restrict__ dz) {
  const long long total = (long long)n * kFeat;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / kFeat, k = e % kFeat;
    const float x = __bfloat162float(feat[r * ldf + k]);
    dz[e] = __float2bfloat16_rn(x > 0.0f ? dfeat[e] : 0.0f);
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float c1, float c2,
                       float eps) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.0f - b1) * gi;
    const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void k_to_bf16(const float* __restrict__ in, long long n, bf16* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = __float2bfloat16_rn(in[e]);
}

// ---------------------------------------------------------------- crops
// One block per hypothesis. The centre is the projection of (x, y, middle of
// V(O)'s height range), in double with every operation rounded separately:
// camera point = R_wc^T (p - t_wc) summed in the order 0, 1, 2; pixel
// floor(f (x_c / z_c) + c + 0.5). A pixel's value is
// clamp((z_ref - d) 10 / m, -3, 3) (float, then bfloat16) where the depth d is
// finite and > 0, else -4 (also outside the image and for a centre behind
// the camera or beyond 1e6 pixels).
__global__ void k_crops(Camera cam, const float* __restrict__ xs, const float* __restrict__ ys,
                        const DevMesh* __restrict__ meshes, int n_yaw, const float* const* __restrict__ scene_img,
                        const int32_t* __restrict__ parent_scene, const float* __restrict__ parent_z,
                        const int32_t* __restrict__ hyp_parent, const perch_obj* __restrict__ hyp, long long n_hyp,
                        bf16* __restrict__ crops, int32_t* __restrict__ onehot) {
  __shared__ int s_cu, s_cv, s_ok;
  __shared__ double s_zr;
  const long long h = blockIdx.x;
  if (h >= n_hyp) return;
  const perch_obj o = hyp[h];
  const int par = hyp_parent[h];
  if (threadIdx.x == 0) {
    const DevMesh& m = meshes[o.mesh];
    const double px = (double)xs[o.ix], py = (double)ys[o.iy];
    const double pz = __dmul_rn(__dadd_rn((double)m.vol_zlo, (double)m.vol_zhi), 0.5);
    const double d0 = __dsub_rn(px, (double)cam.twc[0]);
    const double d1 = __dsub_rn(py, (double)cam.twc[1]);
    const double d2 = __dsub_rn(pz, (double)cam.twc[2]);
    double c[3];
    for (int k = 0; k < 3; ++k)
      c[k] = __dadd_rn(__dadd_rn(__dmul_rn((double)cam.Rwc[0 * 3 + k], d0), __dmul_rn((double)cam.Rwc[1 * 3 + k], d1)),
                       __dmul_rn((double)cam.Rwc[2 * 3 + k], d2));
    int ok = c[2] > 0.0;
    double u = 0.0, v = 0.0;
    if (ok) {
      u = __dadd_rn(__dmul_rn((double)cam.fx, __ddiv_rn(c[0], c[2])), (double)cam.cx);
      v = __dadd_rn(__dmul_rn((double)cam.fy, __ddiv_rn(c[1], c[2])), (double)cam.cy);
      ok = fabs(u) < 1e6 && fabs(v) < 1e6;
    }
    s_ok = ok;
    s_cu = ok ? (int)floor(__dadd_rn(u, 0.5)) : 0;
    s_cv = ok ? (int)floor(__dadd_rn(v, 0.5)) : 0;
    s_zr = c[2];
    onehot[h] = (int32_t)o.mesh * n_yaw + o.iyaw;
  }
  __syncthreads();
  const int W = cam.W, H = cam.H;
  const int sc = parent_scene ? parent_scene[par] : 0;
  const float* img = scene_img[sc];
  const float* pz = parent_z + (long long)par * W * H;
  const double zr = s_zr;
  for (int px = threadIdx.x; px < kCrop * kCrop; px += blockDim.x) {
    const int r = s_cv - kCrop / 2 + px / kCrop, c = s_cu - kCrop / 2 + px % kCrop;
    float val[2] = {kMissing, kMissing};
    if (s_ok && r >= 0 && r < H && c >= 0 && c < W) {
      const float d[2] = {img[(long long)r * W + c], pz[(long long)r * W + c]};
      for (int ch = 0; ch < 2; ++ch)
        if (isfinite(d[ch]) && d[ch] > 0.0f) {
          const float t = __double2float_rn(__dmul_rn(__dsub_rn(zr, (double)d[ch]), kScale));
          val[ch] = fminf(fmaxf(t, -kClamp), kClamp);
        }
    }
    *reinterpret_cast<__nv_bfloat162*>(crops + (h * kCrop * kCrop + px) * 2) = __floats2bfloat162_rn(val[0], val[1]);
  }
}

int grid_for(long long n, int threads = 256) {
  return (int)std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, 152LL * 16));
}

}  // namespace

// ---------------------------------------------------------------- network object
struct perch_cnn {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  int n_onehot = 0, onehot_pad = 0, Kf = 0, max_batch = 0;
  long long step = 0;
  // FP32 master layout: conv weights [Cout][Kp], FC1 [96][Kf] (the bfloat16
  // region, contiguous), then conv biases, FC1 bias, FC2 weights, FC2 bias
  long long off_w[kConvs], off_f1, n_w16, off_b[kConvs], off_fb1, off_f2, off_fb2, n_total;
  DevBuf master, grad, adam_m, adam_v, w16;
  // batch buffers
  DevBuf col[kConvs], act[kConvs], feat, h1, err_buf, pred_buf, loss_buf;
  DevBuf dz1, dfeat, dz, dcol, part, bpart;
  bool params_set = false;
  // forward 3x3 convolutions 2-4 on tcgen05 (else mma.sync); tc_err: the
  // tcgen05 kernel's wait-gave-up flag (device int)
  bool tensor_tc = false;
  DevBuf tc_err;

  int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return code;
  }
  int cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return PERCH_OK;
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return fail(PERCH_E_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(PERCH_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
  }
  std::vector<DevBuf*> buffers() {
    std::vector<DevBuf*> v = {&master, &grad, &adam_m, &adam_v, &w16, &feat, &h1, &err_buf, &pred_buf,
                              &loss_buf, &dz1, &dfeat, &dz, &dcol, &part, &bpart, &tc_err};
    for (int l = 0; l < kConvs; ++l) {
      v.push_back(&col[l]);
      v.push_back(&act[l]);
    }
    return v;
  }
  void layout() {
    long long o = 0;
    for (int l = 0; l < kConvs; ++l) {
      off_w[l] = o;
      o += (long long)kCout[l] * kp_of(l);
    }
    off_f1 = o;
    o += (long long)kHidden * Kf;
    n_w16 = o;
    for (int l = 0; l < kConvs; ++l) {
      off_b[l] = o;
      o += kCout[l];
    }
    off_fb1 = o;
    o += kHidden;
    off_f2 = o;
    o += kHidden;
    off_fb2 = o;
    o += 4;
    n_total = o;
  }
  long long n_params() const {  // unpadded count, the packed order of the ABI
    long long n = 0;
    for (int l = 0; l < kConvs; ++l) n += (long long)kCout[l] * 9 * kCin[l] + kCout[l];
    return n + (long long)kHidden * (kFeat + n_onehot) + kHidden + kHidden + 1;
  }
  // packed (ABI) index <-> padded master index, in the packed order
  template <typename F>
  void for_each_param(F f) const {
    long long q = 0;
    for (int l = 0; l < kConvs; ++l) {
      const int K = 9 * kCin[l], Kp = kp_of(l);
      for (int o = 0; o < kCout[l]; ++o)
        for (int k = 0; k < K; ++k) f(q++, off_w[l] + (long long)o * Kp + k);
      for (int o = 0; o < kCout[l]; ++o) f(q++, off_b[l] + o);
    }
    for (int o = 0; o < kHidden; ++o)
      for (int k = 0; k < kFeat + n_onehot; ++k) f(q++, off_f1 + (long long)o * Kf + k);
    for (int o = 0; o < kHidden; ++o) f(q++, off_fb1 + o);
    for (int o = 0; o < kHidden; ++o) f(q++, off_f2 + o);
    f(q++, off_fb2);
  }
  int ensure_batch(int n);
  int refresh_weights();
  int forward(const bf16* crops, const int32_t* onehot, int n, float* pred, const float* target);
  int backward(const bf16* crops, int n);
};

#define CK_CTX(expr, what)                    \
  do {                                        \
    int rc_ = ctx->cuda((expr), what);        \
    if (rc_ != PERCH_OK) return rc_;          \
  } while (0)

#define CKN(expr, what)                       \
  do {                                        \
    int rc_ = net->cuda((expr), what);        \
    if (rc_ != PERCH_OK) return rc_;          \
  } while (0)

int perch_cnn::ensure_batch(int n) {
  perch_cnn* net = this;
  const long long N = std::max(n, 32);
  for (int l = 0; l < kConvs; ++l) {
    const long long Ho = kHin[l] / kStride[l];
    if (l == 0) CKN(col[0].ensure(2 * N * Ho * Ho * kp_of(0)), "alloc im2col");
    if (l < kConvs - 1) CKN(act[l].ensure(2 * N * Ho * Ho * kCout[l]), "alloc activations");
  }
  CKN(feat.ensure(2 * N * Kf), "alloc");
  CKN(h1.ensure(2 * N * kHidden), "alloc");
  CKN(err_buf.ensure(4 * N), "alloc");
  CKN(pred_buf.ensure(4 * N), "alloc");
  CKN(loss_buf.ensure(16), "alloc");
  return PERCH_OK;
}

int perch_cnn::refresh_weights() {
  perch_cnn* net = this;
  CKN(w16.ensure(2 * n_w16), "alloc");
  k_to_bf16<<<grid_for(n_w16), 256, 0, stream>>>(master.as<float>(), n_w16, w16.as<bf16>());
  CKN(cudaGetLastError(), "cast kernel");
  return PERCH_OK;
}

// Forward pass of n <= max_batch crops; with a target also the per-sample
// errors (for the backward pass).
int perch_cnn::forward(const bf16* crops, const int32_t* onehot, int n, float* pred, const float* target) {
  perch_cnn* net = this;
  int rc = ensure_batch(n);
  if (rc) return rc;
  const bf16* x = crops;
  for (int l = 0; l < kConvs; ++l) {
    const int H = kHin[l], s = kStride[l], Ho = H / s, Kp = kp_of(l);
    const long long M = (long long)n * Ho * Ho;
    GemmArgs p{};
    if (l == 0) {  // two input channels: explicit rows of 32 columns
      k_im2col_c2<<<grid_for(M), 256, 0, stream>>>(reinterpret_cast<const uint32_t*>(x), n, H, H,
                                                   col[0].as<uint4>());
      CKN(cudaGetLastError(), "im2col kernel");
      p.A = col[0].as<bf16>();
      p.lda = Kp;
    } else {  // implicit im2col from the NHWC activations
      p.A = x;
      set_conv(p, l);
    }
    p.B = w16.as<bf16>() + off_w[l];
    p.ldb = Kp;
    p.M = (int)M;
    p.N = kCout[l];
    p.K = Kp;
    p.Ksplit = Kp;
    p.bias = master.as<float>() + off_b[l];
    if (l < kConvs - 1) {
      p.Cb = act[l].as<bf16>();
      p.ldc = kCout[l];
    } else {  // straight into the FC input rows: crop m / 64, position m % 64
      p.Cb = feat.as<bf16>();
      p.ldc = kCout[l];
      p.grp = Ho * Ho;
      p.ldg = Kf;
    }
    if (l == 0)
      CKN(gemm<EPI_BIAS_RELU>(p, 1, stream), "conv gemm");
    else if (tensor_tc)
      CKN(conv_tc(p, tc_err.as<int>(), stream), "conv tcgen05");
    else
      CKN((gemm<EPI_BIAS_RELU, true, true, 1>(p, 1, stream)), "conv gemm");
    x = l < kConvs - 1 ? act[l].as<bf16>() : nullptr;
  }
  k_onehot<<<grid_for((long long)n * onehot_pad), 256, 0, stream>>>(onehot, n, n, onehot_pad, Kf, feat.as<bf16>());
  CKN(cudaGetLastError(), "one-hot kernel");
  // FC1: few output tiles over a long K, so split K and finish bias + ReLU in a second pass
  GemmArgs p{};
  p.A = feat.as<bf16>();
  p.lda = Kf;
  p.B = w16.as<bf16>() + off_f1;
  p.ldb = Kf;
  p.M = n;
  p.N = kHidden;
  p.K = Kf;
  const int S = choose_splits(n, kHidden, Kf, &p.Ksplit);
  CKN(part.ensure(4 * (size_t)S * n * kHidden), "alloc");
  p.Cf = part.as<float>();
  p.ldc = kHidden;
  p.split_stride = (long long)n * kHidden;
  CKN(gemm<EPI_F32>(p, S, stream), "fc1 gemm");
  k_splits_bias_relu<<<grid_for((long long)n * kHidden), 256, 0, stream>>>(
      part.as<float>(), S, n, kHidden, master.as<float>() + off_fb1, h1.as<bf16>());
  CKN(cudaGetLastError(), "fc1 epilogue kernel");
  k_fc2<<<(n * 32 + 255) / 256, 256, 0, stream>>>(h1.as<bf16>(), master.as<float>() + off_f2,
                                                   master.as<float>() + off_fb2, n, pred, target, err_buf.as<float>());
  CKN(cudaGetLastError(), "fc2 kernel");
  return PERCH_OK;
}

// Backward pass after forward(..., target); n a multiple of 32. Fills `grad`.
int perch_cnn::backward(const bf16* crops, int n) {
  perch_cnn* net = this;
  const long long N = n;
  float* G = grad.as<float>();
  CKN(dz1.ensure(2 * N * kHidden), "alloc");
  CKN(dfeat.ensure(4 * N * kFeat), "alloc");
  long long max_mk = 0, max_part = 0, max_bpart = 0;
  for (int l = 0; l < kConvs; ++l) {
    const long long Ho = kHin[l] / kStride[l], M = N * Ho * Ho;
    max_mk = std::max(max_mk, M * std::max(kp_of(l), kCout[l]));
    int ks;
    const int S = choose_splits(kCout[l], kp_of(l), (int)M, &ks);
    max_part = std::max(max_part, (long long)S * kCout[l] * kp_of(l));
    max_bpart = std::max(max_bpart, 2048LL * kCout[l]);
  }
  max_bpart = std::max(max_bpart, 2048LL * kHidden);
  CKN(dz.ensure(2 * max_mk), "alloc");
  CKN(dcol.ensure(2 * max_mk), "alloc");
  CKN(part.ensure(4 * max_part), "alloc");
  CKN(bpart.ensure(4 * max_bpart), "alloc");
  auto bias_grad = [&](const bf16* d, long long M, int C, float* out) -> int {
    const int R = (int)std::max<long long>(16, (M + 2047) / 2048);  // at most 2048 blocks
    const int nb = (int)((M + R - 1) / R);
    k_col_sum<<<nb, 256, 0, stream>>>(d, M, C, R, bpart.as<float>());
    k_split_sum_wide<<<(C + 31) / 32, 1024, 0, stream>>>(bpart.as<float>(), nb, C, out);
    return net->cuda(cudaGetLastError(), "bias gradient kernels");
  };
  // FC2 and the loss
  k_fc2_loss<<<1, 256, 0, stream>>>(err_buf.as<float>(), n, G + off_fb2, loss_buf.as<float>());
  k_fc2_wgrad<<<kHidden, 256, 0, stream>>>(h1.as<bf16>(), err_buf.as<float>(), n, G + off_f2);
  k_fc2_dz1<<<grid_for(N * kHidden), 256, 0, stream>>>(h1.as<bf16>(), master.as<float>() + off_f2,
                                                       err_buf.as<float>(), n, dz1.as<bf16>());
  CKN(cudaGetLastError(), "fc2 backward kernels");
  // FC1: dW = dz1^T feat (reduction over the batch, both operands batch-major),
  // db = column sums of dz1, dfeat = dz1 W (W read as [K][N])
  {
    GemmArgs p{};
    p.A = dz1.as<bf16>();
    p.lda = kHidden;
    p.B = feat.as<bf16>();
    p.ldb = Kf;
    p.M = kHidden;
    p.N = Kf;
    p.K = n;
    p.Ksplit = n;
    p.Cf = G + off_f1;
    p.ldc = Kf;
    CKN((gemm<EPI_F32, false, false>(p, 1, stream)), "fc1 weight-gradient gemm");
  }
  if (int rc = bias_grad(dz1.as<bf16>(), N, kHidden, G + off_fb1)) return rc;
  {
    GemmArgs p{};
    p.A = dz1.as<bf16>();
    p.lda = kHidden;
    p.B = w16.as<bf16>() + off_f1;  // columns 0 .. kFeat-1 of W: the conv features only
    p.ldb = Kf;
    p.M = n;
    p.N = kFeat;
    p.K = kHidden;
    p.Ksplit = kHidden;
    p.Cf = dfeat.as<float>();
    p.ldc = kFeat;
    CKN((gemm<EPI_F32, true, false>(p, 1, stream)), "fc1 data-gradient gemm");
  }
  bf16* cur = dz.as<bf16>();   // gradient of the current layer's output
  bf16* nxt = dcol.as<bf16>();  // receives the gradient of its input
  k_feat_relu_grad<<<grid_for(N * kFeat), 256, 0, stream>>>(dfeat.as<float>(), feat.as<bf16>(), Kf, n,
                                                             cur);
  CKN(cudaGetLastError(), "relu gradient kernel");
  for (int l = kConvs - 1; l >= 0; --l) {
    const int H = kHin[l], s = kStride[l], Ho = H / s, Kp = kp_of(l), Co = kCout[l];
    const long long M = N * Ho * Ho;
    if (int rc = bias_grad(cur, M, Co, G + off_b[l])) return rc;
    // dW = dz^T col: both operands pixel-major, split along the pixel reduction,
    // partials summed in order
    {
      GemmArgs p{};
      p.A = cur;
      p.lda = Co;
      p.M = Co;
      p.N = Kp;
      p.K = (int)M;
      const int S = choose_splits(Co, Kp, (int)M, &p.Ksplit);
      p.Cf = part.as<float>();
      p.ldc = Kp;
      p.split_stride = (long long)Co * Kp;
      if (l == 0) {
        p.B = col[0].as<bf16>();
        p.ldb = Kp;
        CKN((gemm<EPI_F32, false, false>(p, S, stream)), "conv weight-gradient gemm");
      } else {  // implicit im2col of this layer's input
        p.B = act[l - 1].as<bf16>();
        set_conv(p, l);
        CKN((gemm<EPI_F32, false, false, 2>(p, S, stream)), "conv weight-gradient gemm");
      }
      k_split_sum_wide<<<(unsigned)((Co * Kp + 31) / 32), 256, 0, stream>>>(part.as<float>(), S,
                                                                             (long long)Co * Kp, G + off_w[l]);
      CKN(cudaGetLastError(), "split sum kernel");
    }
    if (l == 0) break;
    // data gradient of this layer's input, ReLU mask applied: one implicit
    // GEMM per parity class of the input pixels (1, 2, 2 or 4 taps), written
    // straight into the other gradient buffer
    for (int ph = 0; ph < 2; ++ph)
      for (int pw = 0; pw < 2; ++pw) {
        GemmArgs p{};
        p.A = cur;
        p.B = w16.as<bf16>() + off_w[l];
        p.M = (int)M;  // the class has as many pixels as the layer output
        p.N = kCin[l];
        p.ntw = pw ? 2 : 1;
        p.K = (ph ? 2 : 1) * p.ntw * Co;
        p.Ksplit = p.K;
        p.par_h = ph;
        p.par_w = pw;
        p.dg_lg_ho = ilog2(Ho);
        p.dg_lg_co = ilog2(Co);
        p.lg_c = p.dg_lg_co;
        p.dg_H = H;
        p.dg_cin = kCin[l];
        p.dg_kp = Kp;
        p.mask = act[l - 1].as<bf16>();
        p.Cb = nxt;
        CKN((gemm<EPI_DGRAD, true, false, 3>(p, 1, stream)), "conv data-gradient gemm");
      }
    std::swap(cur, nxt);
  }
  (void)crops;
  return PERCH_OK;
}

int net_predict(perch_ctx* ctx, perch_cnn* net, const perch_obj* parents, int parent_stride, const int32_t* plen,
                const int32_t* pscene, int n_par, const int32_t* hyp_parent, const perch_obj* hyp, long long n_hyp,
                float* pred_host) {
  if (n_hyp == 0) return PERCH_OK;
  CK_CTX(ctx->net_crops.ensure(2 * (size_t)kCrop * kCrop * 2 * n_hyp), "alloc crops");
  CK_CTX(ctx->net_onehot.ensure(4 * (size_t)n_hyp), "alloc");
  CK_CTX(ctx->net_pred.ensure(4 * (size_t)n_hyp), "alloc");
  int rc = perch_cnn_crops(ctx, parents, parent_stride, plen, pscene, n_par, hyp_parent, hyp, n_hyp,
                           ctx->net_crops.as<uint16_t>(), ctx->net_onehot.as<int32_t>());
  if (rc) return rc;
  rc = perch_cnn_forward(net, ctx->net_crops.as<uint16_t>(), ctx->net_onehot.as<int32_t>(), n_hyp,
                         ctx->net_pred.as<float>());
  if (rc) return ctx->fail(rc, "learned heuristic: %s", net->err.c_str());
  CK_CTX(cudaMemcpyAsync(pred_host, ctx->net_pred.p, 4 * (size_t)n_hyp, cudaMemcpyDeviceToHost, net->stream),
         "copy predictions");
  CK_CTX(cudaStreamSynchronize(net->stream), "learned heuristic");
  return PERCH_OK;
}

// ---------------------------------------------------------------- C ABI
extern "C" {

int perch_cnn_create(perch_cnn** out, int device, void* cuda_stream, int32_t n_onehot, int32_t max_batch) {
  if (!out) return PERCH_E_ARG;
  *out = nullptr;
  if (n_onehot < 1 || n_onehot > 65536 || max_batch < 32 || max_batch > 1024 || max_batch % 32) return PERCH_E_ARG;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return PERCH_E_CUDA;
  }
  perch_cnn* net = new perch_cnn;
  net->device = device;
  net->n_onehot = n_onehot;
  net->onehot_pad = round32(n_onehot);
  net->Kf = kFeat + net->onehot_pad;
  net->max_batch = max_batch;
  net->layout();
  if (cuda_stream) {
    net->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete net;
      return PERCH_E_CUDA;
    }
    net->own_stream = true;
  }
  const size_t bytes = 4 * (size_t)net->n_total;
  bool ok = net->master.ensure(bytes) == cudaSuccess && net->grad.ensure(bytes) == cudaSuccess &&
            net->adam_m.ensure(bytes) == cudaSuccess && net->adam_v.ensure(bytes) == cudaSuccess &&
            net->tc_err.ensure(16) == cudaSuccess && cudaMemsetAsync(net->tc_err.p, 0, 16, net->stream) == cudaSuccess;
  ok = ok && cudaMemsetAsync(net->master.p, 0, bytes, net->stream) == cudaSuccess &&
       cudaMemsetAsync(net->grad.p, 0, bytes, net->stream) == cudaSuccess &&
       cudaMemsetAsync(net->adam_m.p, 0, bytes, net->stream) == cudaSuccess &&
       cudaMemsetAsync(net->adam_v.p, 0, bytes, net->stream) == cudaSuccess;
  ok = ok && net->refresh_weights() == PERCH_OK && cudaStreamSynchronize(net->stream) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    for (DevBuf* b : net->buffers()) b->release();
    if (net->own_stream) cudaStreamDestroy(net->stream);
    delete net;
    return PERCH_E_CUDA;
  }
  *out = net;
  return PERCH_OK;
}

int perch_cnn_destroy(perch_cnn* net) {
  if (!net) return PERCH_OK;
  cudaSetDevice(net->device);
  cudaStreamSynchronize(net->stream);
  for (DevBuf* b : net->buffers()) b->release();
  if (net->own_stream) cudaStreamDestroy(net->stream);
  delete net;
  return PERCH_OK;
}

const char* perch_cnn_last_error(const perch_cnn* net) { return net ? net->err.c_str() : "null network"; }

int perch_cnn_set_tensor_path(perch_cnn* net, int32_t path) {
  if (!net) return PERCH_E_ARG;
  if (path != 0 && path != 1) return net->fail(PERCH_E_ARG, "tensor path must be 0 (mma.sync) or 1 (tcgen05)");
  net->tensor_tc = path == 1;
  return PERCH_OK;
}

int perch_cnn_tensor_status(perch_cnn* net, int32_t* path, int32_t* waits_gave_up) {
  if (!net) return PERCH_E_ARG;
  if (cudaSetDevice(net->device) != cudaSuccess) return net->cuda(cudaGetLastError(), "cudaSetDevice");
  int e = 0;
  int rc = net->cuda(cudaStreamSynchronize(net->stream), "stream");
  if (rc) return rc;
  rc = net->cuda(cudaMemcpy(&e, net->tc_err.p, sizeof e, cudaMemcpyDeviceToHost), "read flag");
  if (rc) return rc;
  if (path) *path = net->tensor_tc ? 1 : 0;
  if (waits_gave_up) *waits_gave_up = e;
  return PERCH_OK;
}

int perch_cnn_param_count(const perch_cnn* net, int64_t* n) {
  if (!net || !n) return PERCH_E_ARG;
  *n = net->n_params();
  return PERCH_OK;
}

int perch_cnn_set_params(perch_cnn* net, const float* params, int64_t n) {
  if (!net) return PERCH_E_ARG;
  net->err.clear();
  if (!params || n != net->n_params()) return net->fail(PERCH_E_ARG, "expected %lld parameters", net->n_params());
  CKN(cudaSetDevice(net->device), "cudaSetDevice");
  std::vector<float> h((size_t)net->n_total, 0.0f);
  net->for_each_param([&](long long q, long long i) { h[i] = params[q]; });
  const size_t bytes = 4 * (size_t)net->n_total;
  CKN(cudaMemcpyAsync(net->master.p, h.data(), bytes, cudaMemcpyHostToDevice, net->stream), "copy parameters");
  CKN(cudaMemsetAsync(net->adam_m.p, 0, bytes, net->stream), "memset");
  CKN(cudaMemsetAsync(net->adam_v.p, 0, bytes, net->stream), "memset");
  net->step = 0;
  int rc = net->refresh_weights();
  if (rc) return rc;
  CKN(cudaStreamSynchronize(net->stream), "set parameters");
  net->params_set = true;
  return PERCH_OK;
}

int perch_cnn_get_params(perch_cnn* net, float* params, int64_t n) {
  if (!net) return PERCH_E_ARG;
  net->err.clear();
  if (!params || n != net->n_params()) return net->fail(PERCH_E_ARG, "expected %lld parameters", net->n_params());
  CKN(cudaSetDevice(net->device), "cudaSetDevice");
  std::vector<float> h((size_t)net->n_total);
  CKN(cudaMemcpyAsync(h.data(), net->master.p, 4 * h.size(), cudaMemcpyDeviceToHost, net->stream), "copy");
  CKN(cudaStreamSynchronize(net->stream), "get parameters");
  net->for_each_param([&](long long q, long long i) { params[q] = h[i]; });
  return PERCH_OK;
}

int perch_cnn_forward(perch_cnn* net, const uint16_t* crops, const int32_t* onehot, int64_t n, float* pred) {
  if (!net) return PERCH_E_ARG;
  net->err.clear();
  if (n < 0 || (n > 0 && (!crops || !onehot || !pred))) return net->fail(PERCH_E_ARG, "bad arguments");
  CKN(cudaSetDevice(net->device), "cudaSetDevice");
  for (int64_t b = 0; b < n; b += net->max_batch) {
    const int nb = (int)std::min<int64_t>(net->max_batch, n - b);
    int rc = net->forward(reinterpret_cast<const bf16*>(crops) + b * 2 * kCrop * kCrop, onehot + b, nb, pred + b,
                          nullptr);
    if (rc) return rc;
  }
  return PERCH_OK;
}

int perch_cnn_gradients(perch_cnn* net, const uint16_t* crops, const int32_t* onehot, const float* target, int32_t n,
                        float* grads, float* loss, float* pred) {
  if (!net) return PERCH_E_ARG;
  net->err.clear();
  if (!crops || !onehot || !target || n < 32 || n > net->max_batch || n % 32)
    return net->fail(PERCH_E_ARG, "need device crops / one-hot / targets and 32 <= n <= %d, n %% 32 == 0",
                     net->max_batch);
  CKN(cudaSetDevice(net->device), "cudaSetDevice");
  int rc = net->ensure_batch(n);
  if (rc) return rc;
  rc = net->forward(reinterpret_cast<const bf16*>(crops), onehot, n, net->pred_buf.as<float>(), target);
  if (rc) return rc;
  rc = net->backward(reinterpret_cast<const bf16*>(crops), n);
  if (rc) return rc;
  if (grads) {
    std::vector<float> h((size_t)net->n_total);
    CKN(cudaMemcpyAsync(h.data(), net->grad.p, 4 * h.size(), cudaMemcpyDeviceToHost, net->stream), "copy");
    CKN(cudaStreamSynchronize(net->stream), "gradients");
    net->for_each_param([&](long long q, long long i) { grads[q] = h[i]; });
  }
  if (loss) CKN(cudaMemcpyAsync(loss, net->loss_buf.p, 4, cudaMemcpyDeviceToHost, net->stream), "copy");
  if (pred) CKN(cudaMemcpyAsync(pred, net->pred_buf.p, 4 * (size_t)n, cudaMemcpyDeviceToHost, net->stream), "copy");
  CKN(cudaStreamSynchronize(net->stream), "gradients");
  return PERCH_OK;
}

int perch_cnn_train_step(perch_cnn* net, const uint16_t* crops, const int32_t* onehot, const float* target,
                         int32_t n, float lr, float* loss) {
  if (!net) return PERCH_E_ARG;
  net->err.clear();
  if (!crops || !onehot || !target || n < 32 || n > net->max_batch || n % 32 || !(lr > 0.0f))
    return net->fail(PERCH_E_ARG, "need device crops / one-hot / targets, 32 <= n <= %d, n %% 32 == 0, lr > 0",
                     net->max_batch);
  CKN(cudaSetDevice(net->device), "cudaSetDevice");
  int rc = net->forward(reinterpret_cast<const bf16*>(crops), onehot, n, net->pred_buf.as<float>(), target);
  if (rc) return rc;
  rc = net->backward(reinterpret_cast<const bf16*>(crops), n);
  if (rc) return rc;
  net->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - std::pow((double)b1, (double)net->step));
  const float c2 = (float)(1.0 - std::pow((double)b2, (double)net->step));
  k_adam<<<grid_for(net->n_total), 256, 0, net->stream>>>(net->master.as<float>(), net->grad.as<float>(),
                                                           net->adam_m.as<float>(), net->adam_v.as<float>(),
                                                           net->n_total, lr, b1, b2, c1, c2, 1e-8f);
  CKN(cudaGetLastError(), "adam kernel");
  rc = net->refresh_weights();
  if (rc) return rc;
  if (loss) CKN(cudaMemcpyAsync(loss, net->loss_buf.p, 4, cudaMemcpyDeviceToDevice, net->stream), "copy loss");
  return PERCH_OK;
}

int perch_cnn_crops(perch_ctx* ctx, const perch_obj* parents, int32_t parent_stride, const int32_t* parent_len,
                    const int32_t* parent_scene, int32_t n_par, const int32_t* hyp_parent, const perch_obj* hyp,
                    int64_t n_hyp, uint16_t* crops, int32_t* onehot) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!ctx->has_obs) return ctx->fail(PERCH_E_STATE, "set an observation first");
  if (n_hyp < 0 || n_hyp > 0x7fffffffLL) return ctx->fail(PERCH_E_ARG, "n_hyp out of range");
  if (n_hyp == 0) return PERCH_OK;
  if (!parent_len || !hyp_parent || !hyp || !crops || !onehot || n_par < 1 || parent_stride < 0 ||
      (parent_stride > 0 && !parents))
    return ctx->fail(PERCH_E_ARG, "null pointer or bad sizes");
  if (n_par > 65535 || (long long)n_par * std::max(parent_stride, 1) > 65535)
    return ctx->fail(PERCH_E_ARG, "too many parents in one batch (n_par x stride <= 65535)");
  auto bad = [&](const perch_obj& o) {
    return o.mesh >= ctx->n_mesh || o.ix < 0 || o.ix >= ctx->nx || o.iy < 0 || o.iy >= ctx->ny ||
           o.iyaw >= ctx->n_yaw;
  };
  for (int i = 0; i < n_par; ++i) {
    if (parent_len[i] < 0 || parent_len[i] > parent_stride)
      return ctx->fail(PERCH_E_ARG, "parent %d: length %d outside [0, stride]", i, parent_len[i]);
    if (parent_scene && (parent_scene[i] < 0 || parent_scene[i] >= (int)ctx->scenes.size()))
      return ctx->fail(PERCH_E_ARG, "parent %d: scene %d not set", i, parent_scene[i]);
    for (int k = 0; k < parent_len[i]; ++k)
      if (bad(parents[(long long)i * parent_stride + k])) return ctx->fail(PERCH_E_ARG, "parent %d: bad object", i);
  }
  for (long long h = 0; h < n_hyp; ++h)
    if (hyp_parent[h] < 0 || hyp_parent[h] >= n_par || bad(hyp[h]))
      return ctx->fail(PERCH_E_ARG, "hypothesis %lld: bad parent or object", h);
  perch_ctx* c = ctx;
  auto ck = [c](cudaError_t e, const char* what) { return c->cuda(e, what); };
  int rc;
  if ((rc = ck(cudaSetDevice(ctx->device), "cudaSetDevice"))) return rc;
  const size_t npx = (size_t)ctx->cam.W * ctx->cam.H;
  const size_t pbytes = sizeof(perch_obj) * std::max<size_t>((size_t)n_par * parent_stride, 1);
  if ((rc = ck(ctx->parent_z.ensure(4 * npx * n_par), "alloc parent z-buffers"))) return rc;
  if ((rc = ck(ctx->b_parents.ensure(pbytes), "alloc"))) return rc;
  if ((rc = ck(ctx->b_plen.ensure(8 * (size_t)n_par), "alloc"))) return rc;
  if ((rc = ck(ctx->b_hp.ensure(4 * (size_t)n_hyp), "alloc"))) return rc;
  if ((rc = ck(ctx->b_hyp.ensure(sizeof(perch_obj) * (size_t)n_hyp), "alloc"))) return rc;
  int32_t* d_plen = ctx->b_plen.as<int32_t>();
  cudaStream_t s = ctx->stream;
  if (parent_stride > 0 &&
      (rc = ck(cudaMemcpyAsync(ctx->b_parents.p, parents, sizeof(perch_obj) * (size_t)n_par * parent_stride,
                               cudaMemcpyHostToDevice, s), "copy")))
    return rc;
  if ((rc = ck(cudaMemcpyAsync(d_plen, parent_len, 4 * (size_t)n_par, cudaMemcpyHostToDevice, s), "copy"))) return rc;
  if (parent_scene &&
      (rc = ck(cudaMemcpyAsync(d_plen + n_par, parent_scene, 4 * (size_t)n_par, cudaMemcpyHostToDevice, s), "copy")))
    return rc;
  if ((rc = ck(cudaMemcpyAsync(ctx->b_hp.p, hyp_parent, 4 * (size_t)n_hyp, cudaMemcpyHostToDevice, s), "copy")))
    return rc;
  if ((rc = ck(cudaMemcpyAsync(ctx->b_hyp.p, hyp, sizeof(perch_obj) * (size_t)n_hyp, cudaMemcpyHostToDevice, s),
               "copy")))
    return rc;
  if ((rc = ck(launch_fill_u32(ctx->parent_z.as<uint32_t>(), kInfBits, (long long)npx * n_par, s), "clear")))
    return rc;
  Batch b;
  std::memset(&b, 0, sizeof b);
  b.parents = ctx->b_parents.as<perch_obj>();
  b.parent_stride = std::max(parent_stride, 1);  // stride 0: every parent is empty
  b.parent_len = d_plen;
  b.n_par = n_par;
  b.parent_z = ctx->parent_z.as<float>();
  if ((rc = ck(launch_render_parents(ctx->cam, ctx->geometry(), b, ctx->max_chunks, nullptr, s), "render parents")))
    return rc;
  k_crops<<<(unsigned)n_hyp, 256, 0, s>>>(ctx->cam, ctx->xs.as<float>(), ctx->ys.as<float>(),
                                          ctx->meshes.as<DevMesh>(), ctx->n_yaw, ctx->d_scene_img.as<const float*>(),
                                          parent_scene ? d_plen + n_par : nullptr, ctx->parent_z.as<float>(),
                                          ctx->b_hp.as<int32_t>(), ctx->b_hyp.as<perch_obj>(), n_hyp,
                                          reinterpret_cast<bf16*>(crops), onehot);
  if ((rc = ck(cudaGetLastError(), "crop kernel"))) return rc;
  return ck(cudaStreamSynchronize(s), "crops");
}

int perch_set_heuristic_net(perch_ctx* ctx, perch_cnn* net, int32_t n_candidates) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (net && net->n_onehot < ctx->n_mesh * ctx->n_yaw)
    return ctx->fail(PERCH_E_ARG, "network one-hot width %d < meshes x yaws %d", net->n_onehot,
                     ctx->n_mesh * ctx->n_yaw);
  if (n_candidates < 1 || n_candidates > 4096) return ctx->fail(PERCH_E_ARG, "n_candidates outside [1, 4096]");
  ctx->net = net;
  ctx->net_candidates = n_candidates;
  return PERCH_OK;
}

}  // extern "C"
