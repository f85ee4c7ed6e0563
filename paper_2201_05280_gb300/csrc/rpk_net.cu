// Learned surrogate network: a 1-D convolutional operator on the moment fields
// of quasi-1-D tubes, with forward, backward and Adam in hand-written kernels.
// The paper has no learned component.
//
// Architecture (fine sequence of L points, L a multiple of R = 4):
//   unshuffle (L, Cin) -> (L/4, 4 Cin)   [a reshape of the position-major layout]
//   lift      conv k=1, 4 Cin -> C, bias
//   B blocks  h <- h + conv5(relu(conv5(relu(h))))   (C -> C, zero padding)
//   head      conv k=1 of relu(h), C -> 4 Cout, bias
//   shuffle   (L/4, 4 Cout) -> (L, Cout)
// Tensors are FP32 in memory, position-major ([position][channel]); every
// contraction runs on the tensor cores with BF16 operands (converted while a
// tile is staged in shared memory) and FP32 accumulation (mma.sync m16n8k16).
//
//   k_conv     out[q][m] = (sum_{t,j} A[m][t][j] * act(X[q + s (t - c)][j]) + bias)
//              x (mask > 0) + residual; s = +1 forward, s = -1 input gradient
//              (A = W transposed per tap), zero outside each sequence
//   k_conv_dw  dW[o][t][i] += sum_q dY[q][o] * act(X[q + t - c][i])  (split over q)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "rpk_internal.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 32, kPadK = 8;  // tile sizes; smem row padding
constexpr int kThreads = 128;                        // 4 warps: 2 (m) x 2 (n), 32 x 32 each
constexpr int R = 4, K5 = 5;

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
  return (uint32_t)(*reinterpret_cast<const uint16_t*>(&x)) |
         ((uint32_t)(*reinterpret_cast<const uint16_t*>(&y)) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct ConvArgs {
  const __nv_bfloat16* A;  // [M][taps][Kc]
  const float* X;          // [npos][Kc], position-major
  float* out;              // [npos][M]
  const float* bias;       // [M] or null
  const float* res;        // [npos][M] added, or null
  const float* mask;       // [npos][M]: out *= (mask > 0), or null
  const int2* qseq;        // per position (first position, length) of its sequence, or null
  int M, Kc, taps, sgn, relu_in;
  int npos, seq_len;       // seq_len: common sequence length when qseq is null
};

// One warp-tile step: 2 x 4 mma over one k16 slice of the staged tiles.
__device__ __forceinline__ void warp_mma(const uint16_t (*As)[BK + kPadK],
                                         const uint16_t (*Bs)[BK + kPadK], int wm, int wn,
                                         int k16, float (&acc)[2][4][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t a[2][4], b[4][2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int r = wm * 32 + i * 16 + g;
    a[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][k16 + 2 * t]);
    a[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][k16 + 2 * t]);
    a[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][k16 + 2 * t + 8]);
    a[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][k16 + 2 * t + 8]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int n = wn * 32 + j * 8 + g;
    b[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[n][k16 + 2 * t]);
    b[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[n][k16 + 2 * t + 8]);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
}

__global__ void __launch_bounds__(kThreads) k_conv(ConvArgs P) {
  __shared__ __align__(16) uint16_t As[BM][BK + kPadK];
  __shared__ __align__(16) uint16_t Bs[BN][BK + kPadK];
  __shared__ int s_lo[BN], s_len[BN];  // sequence of each position of the tile
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (threadIdx.x < BN) {
    const int q = n0 + threadIdx.x;
    int lo = 0, len = 0;
    if (q < P.npos) {
      if (P.qseq) {
        const int2 v = P.qseq[q];
        lo = v.x;
        len = v.y;
      } else {
        lo = (q / P.seq_len) * P.seq_len;
        len = P.seq_len;
      }
    }
    s_lo[threadIdx.x] = lo;
    s_len[threadIdx.x] = len;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, wm = warp >> 1, wn = warp & 1;
  const int c = (P.taps - 1) / 2;
  const int K = P.taps * P.Kc;
  float acc[2][4][4] = {};
  for (int k0 = 0; k0 < K; k0 += BK) {
    // stage A (m, k) and B (n, k) as bf16
    for (int e = threadIdx.x; e < BM * BK / 2; e += kThreads) {
      const int mm = e / (BK / 2), kk = 2 * (e % (BK / 2));
      const int m = m0 + mm;
      float v0 = 0.f, v1 = 0.f;
      if (m < P.M) {
        const int ka = k0 + kk, kb = ka + 1;
        if (ka < K) v0 = __bfloat162float(P.A[(int64_t)m * K + ka]);
        if (kb < K) v1 = __bfloat162float(P.A[(int64_t)m * K + kb]);
      }
      *reinterpret_cast<uint32_t*>(&As[mm][kk]) = pack_bf16(v0, v1);
    }
    for (int e = threadIdx.x; e < BN * BK / 2; e += kThreads) {
      const int nn = e / (BK / 2), kk = 2 * (e % (BK / 2));
      const int q = n0 + nn;
      float v[2] = {0.f, 0.f};
      if (q < P.npos) {
        const int lo = s_lo[nn], len = s_len[nn], l = q - lo;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = k0 + kk + h;
          if (k < K) {
            const int t = k / P.Kc, j = k - t * P.Kc;
            const int l2 = l + P.sgn * (t - c);
            if (l2 >= 0 && l2 < len) {
              float x = P.X[((int64_t)lo + l2) * P.Kc + j];
              v[h] = P.relu_in ? fmaxf(x, 0.f) : x;
            }
          }
        }
      }
      *reinterpret_cast<uint32_t*>(&Bs[nn][kk]) = pack_bf16(v[0], v[1]);
    }
    __syncthreads();
    warp_mma(As, Bs, wm, wn, 0, acc);
    warp_mma(As, Bs, wm, wn, 16, acc);
    __syncthreads();
  }
  // epilogue
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int m = m0 + wm * 32 + i * 16 + g + (h >= 2 ? 8 : 0);
        const int q = n0 + wn * 32 + j * 8 + 2 * t + (h & 1);
        if (m < P.M && q < P.npos) {
          const int64_t o = (int64_t)q * P.M + m;
          float v = acc[i][j][h];
          if (P.bias) v += P.bias[m];
          if (P.mask && !(P.mask[o] > 0.f)) v = 0.f;
          if (P.res) v += P.res[o];
          P.out[o] = v;
        }
      }
}

// ---------------------------------------------------------------------------
// Tensor-core (tcgen05) path of the residual-block convolutions: Co = Ci = 128,
// 5 taps. One persistent CTA per SM keeps the layer's BF16 weights in shared
// memory (A: 128 x 640, K-major) and walks over tiles of 128 output positions
// of one sequence. Three roles run concurrently:
//   producers (warps 8-15) load tile i's 132 input rows (positions q0 - 2 ..
//     q0 + 129, every load in flight at once, 9 per thread) into registers
//     while the MMAs of tile i - 1 still read the single input buffer B, then
//     wait for B to be free and store the rows (activation applied, BF16);
//   one issuing thread (warp 8, lane 0) waits for B and for the accumulator
//     i % 2 to be free, issues 40 MMAs (M 128, N 128, K 16) into TMEM columns
//     128 (i % 2) .. + 127 and commits to two mbarriers (B free, accumulator
//     full);
//   the epilogue (warps 0-7; TMEM lane = output channel, lane quadrant
//     warp % 4) writes the tile as four quarters of 32 positions through two
//     16 KB staging buffers in the output's own layout: the residual rows of
//     the next quarter are bulk-copied into the other buffer (cp.async.bulk,
//     completion on an mbarrier) while each thread adds its accumulator
//     column, bias and mask to its elements of this one, and one thread
//     bulk-copies the quarter to the output rows. The epilogue's global
//     traffic is then two bulk copies per quarter instead of 64 loads and 64
//     stores per thread, whose latency had set the tile period.
// The operand of tap t is the staged tile seen from row t (forward) or 4 - t
// (input gradient): in the interleaved no-swizzle layout (rows 16 bytes apart
// inside each 8-column chunk) a row shift is a start-address offset.
constexpr int TC_M = 128, TC_N = 128, TC_KC = 128, TC_TAPS = 5;
constexpr int TC_ROWS = TC_N + TC_TAPS - 1;                // 132 staged rows
constexpr int TC_K = TC_TAPS * TC_KC;                      // 640
constexpr uint32_t TC_A_LBO = TC_M * 16;                   // bytes between 8-wide k chunks of A
// bytes between 8-wide k chunks of B: one row more than staged, so that the
// producers' 16-byte stores of one row's consecutive chunks fall in distinct
// shared-memory banks (2128 / 4 = 532 = 20 mod 32)
constexpr uint32_t TC_B_LBO = (TC_ROWS + 1) * 16;
constexpr uint32_t TC_A_BYTES = (TC_K / 8) * TC_A_LBO;     // 163840
constexpr uint32_t TC_B_BYTES = (TC_KC / 8) * TC_B_LBO;    // 34048
constexpr int TC_QTR = TC_N / 4;                           // positions per staged quarter tile
constexpr uint32_t TC_SQ_BYTES = TC_QTR * TC_M * 4;        // 16384: FP32 rows of a quarter tile
constexpr uint32_t TC_S_BYTES = 2 * TC_SQ_BYTES;           // two staging buffers
constexpr uint32_t TC_S_OFF = TC_A_BYTES + TC_B_BYTES;
constexpr uint32_t TC_BAR_OFF = TC_S_OFF + TC_S_BYTES;
constexpr uint32_t TC_SMEM = TC_BAR_OFF + 128;             // 8 mbarriers + TMEM address
static_assert(TC_SMEM <= 227 * 1024, "tensor-core tiles exceed shared memory");
static_assert(TC_S_OFF % 128 == 0, "the staging buffer is a bulk-copy operand");
constexpr int TC_THREADS = 512;
constexpr int TC_EPI = 256;                                // epilogue threads (warps 0-7)
constexpr int TC_PROD = TC_THREADS - TC_EPI;               // producer threads (warps 8-15)
constexpr int TC_COLS = 2 * TC_N;                          // two accumulators
constexpr long long TC_WAIT_LIMIT = 1ll << 22;             // mbarrier polls before giving up

struct TcArgs {
  const __nv_bfloat16* A;  // [128][5][128]
  const float* X;          // [npos][128]
  float* out;              // [npos][128]
  const float* bias;
  const float* res;
  const float* mask;
  const int4* tiles;       // per tile (q0, count, sequence start, sequence length), or null
  int ntiles, seq_len, tiles_per_seq, sgn, relu_in;
  unsigned* error;         // set to 1 when an mbarrier wait gives up
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start, leading (k-chunk) and stride
// (8-row group) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < TC_WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_tile(const TcArgs& P, int tile, int& q0, int& cnt, int& lo, int& len) {
  if (P.tiles) {
    const int4 d = P.tiles[tile];
    q0 = d.x, cnt = d.y, lo = d.z, len = d.w;
  } else {
    const int sq = tile / P.tiles_per_seq, part = tile - sq * P.tiles_per_seq;
    lo = sq * P.seq_len;
    len = P.seq_len;
    q0 = lo + part * TC_N;
    cnt = min(TC_N, len - part * TC_N);
  }
}

// Barrier 1 among the 256 epilogue threads (the producers never use it).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(TC_EPI) : "memory"); }

// The same barrier, returning whether p holds in every epilogue thread: the
// epilogue warps then leave their loops together and no warp waits at a
// barrier that another has left.
// 16 consecutive accumulator columns of this thread's TMEM lane (32x32b shape)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ bool epi_all(bool p) {
  int r;
  asm volatile(
      "{\n .reg .pred pi, po;\n setp.ne.b32 pi, %1, 0;\n bar.red.and.pred po, 1, %2, pi;\n"
      " selp.b32 %0, 1, 0, po;\n}\n"
      : "=r"(r)
      : "r"((int)p), "n"(TC_EPI)
      : "memory");
  return r != 0;
}

// Bulk copy of the residual rows of quarter q of a tile (positions q0 + 32 q ..)
// into a staging buffer, completing with its byte count on the mbarrier bar.
__device__ __forceinline__ void qtr_load(const TcArgs& P, uint32_t bar, uint32_t dst, int q0, int cnt, int q) {
  const int rows = min(TC_QTR, cnt - q * TC_QTR);
  const uint32_t bytes = (uint32_t)rows * TC_M * 4;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(P.res + (int64_t)(q0 + q * TC_QTR) * TC_M), "r"(bytes), "r"(bar)
               : "memory");
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_conv_tc(TcArgs P) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* sA = tc_smem;
  unsigned char* sB = tc_smem + TC_A_BYTES;
  float* sS = reinterpret_cast<float*>(tc_smem + TC_S_OFF);
  uint64_t* bars = reinterpret_cast<uint64_t*>(tc_smem + TC_BAR_OFF);
  // bars: 0 B full, 1 B free, 2-3 accumulator full, 4-5 accumulator free, 6-7 residual in S[0], S[1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tc_smem + TC_BAR_OFF + 64);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bars)), "r"(TC_PROD) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bars + 1)), "r"(1) : "memory");
    for (int a = 0; a < 2; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bars + 2 + a)), "r"(1) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bars + 4 + a)), "r"(TC_EPI) : "memory");
    }
    for (int q = 0; q < 2; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bars + 6 + q)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weights: chunk c (k = 8c .. 8c + 7) of row m at c * TC_A_LBO + m * 16,
  // copied global -> shared asynchronously (every thread's 20 copies in flight
  // at once, no register round trip)
  for (int e = tid; e < TC_M * (TC_K / 8); e += TC_THREADS) {
    const int m = e % TC_M, c = e / TC_M;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sA + c * TC_A_LBO + m * 16)),
                 "l"(P.A + (int64_t)m * TC_K + 8 * c)
                 : "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB), s_base = smem_u32(sS);
  const uint32_t bar0 = smem_u32(bars);
  bool ok = true;

  if (tid >= TC_EPI) {
    // producers, and the issuing thread
    const int ptid = tid - TC_EPI;
    // 2112 (row, 8-channel chunk) elements, at most 9 per thread; consecutive
    // threads take consecutive 32-byte chunks of a row (coalesced 512-byte rows)
    constexpr int kElems = TC_ROWS * (TC_KC / 8);
    constexpr int kBatch = (kElems + TC_PROD - 1) / TC_PROD;
    static_assert(kBatch * TC_PROD >= kElems, "one batch of loads covers the tile");
    for (int i = 0, tile = blockIdx.x; tile < P.ntiles && ok; ++i, tile += gridDim.x) {
      int q0, cnt, lo, len;
      tc_tile(P, tile, q0, cnt, lo, len);
      // every load of tile i is issued while the MMAs of tile i - 1 still read B
      float4 f[kBatch][2];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int e = ptid + u * TC_PROD;
        const int r = e / (TC_KC / 8), c = e % (TC_KC / 8);
        const int q = q0 - 2 + r;
        f[u][0] = f[u][1] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < kElems && q >= lo && q < lo + len) {
          const float4* src = reinterpret_cast<const float4*>(P.X + (int64_t)q * TC_KC + 8 * c);
          f[u][0] = src[0];
          f[u][1] = src[1];
        }
      }
      // B free: the MMAs of tile i - 1 have completed
      if (i >= 1) ok = __all_sync(0xffffffffu, mbar_wait(bar0 + 8, (i - 1) & 1));
      if (!ok) break;
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int e = ptid + u * TC_PROD;
        if (e >= kElems) break;
        const int r = e / (TC_KC / 8), c = e % (TC_KC / 8);
        float4 f0 = f[u][0], f1 = f[u][1];
        if (P.relu_in) {
          f0.x = fmaxf(f0.x, 0.f), f0.y = fmaxf(f0.y, 0.f), f0.z = fmaxf(f0.z, 0.f), f0.w = fmaxf(f0.w, 0.f);
          f1.x = fmaxf(f1.x, 0.f), f1.y = fmaxf(f1.y, 0.f), f1.z = fmaxf(f1.z, 0.f), f1.w = fmaxf(f1.w, 0.f);
        }
        *reinterpret_cast<uint4*>(sB + c * TC_B_LBO + r * 16) =
            make_uint4(pack_bf16(f0.x, f0.y), pack_bf16(f0.z, f0.w), pack_bf16(f1.x, f1.y),
                       pack_bf16(f1.z, f1.w));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(bar0);  // B full (TC_PROD arrivals)
      if (ptid == 0) {
        // the issuing thread: B staged by all producers, accumulator i % 2 free
        const int acc = i & 1;
        bool go = mbar_wait(bar0, i & 1);
        if (go && i >= 2) go = mbar_wait(bar0 + 8 * (4 + acc), ((i >> 1) - 1) & 1);
        if (go) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d = tmem + (uint32_t)(acc * TC_N);
#pragma unroll 1
          for (int t = 0; t < TC_TAPS; ++t) {
            const int row0 = P.sgn > 0 ? t : TC_TAPS - 1 - t;
#pragma unroll
            for (int s = 0; s < TC_KC / 16; ++s) {
              const uint64_t ad =
                  tc_desc(a_base + (uint32_t)(t * (TC_KC / 8) + 2 * s) * TC_A_LBO, TC_A_LBO, 128);
              const uint64_t bd = tc_desc(b_base + (uint32_t)(2 * s) * TC_B_LBO + (uint32_t)row0 * 16, TC_B_LBO, 128);
              const uint32_t accum = (t | s) ? 1u : 0u;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                  "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(accum)
                  : "memory");
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           bar0 + 8)
                       : "memory");
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           bar0 + 8 * (2 + acc))
                       : "memory");
        } else {
          atomicOr(P.error, 1u);
        }
      }
      __syncwarp();
    }
  } else {
    // epilogue: TMEM lane = output channel m; a tile is written as four
    // quarters of 32 positions through two 16 KB staging buffers (quarter q in
    // S[q % 2]); warps 0-3 take positions 0-15 of a quarter, warps 4-7 16-31.
    // With a residual, the rows of quarter q + 1 are bulk-loaded into the other
    // buffer while quarter q is computed; every quarter leaves as one bulk store.
    const int quad = warp & 3, sub = warp >> 2;
    const int m = quad * 32 + lane;
    const float bm = P.bias ? P.bias[m] : 0.f;
    const uint32_t rbar = bar0 + 8 * 6;  // 6: residual in S[0], 7: residual in S[1]
    int rphase[2] = {0, 0};  // residual copies waited for, per buffer (every thread)
    int rissued[2] = {0, 0};  // residual copies issued, per buffer (thread 0)
    for (int i = 0, tile = blockIdx.x; tile < P.ntiles; ++i, tile += gridDim.x) {
      const int acc = i & 1;
      int q0, cnt, lo, len;
      tc_tile(P, tile, q0, cnt, lo, len);
      const int nq = (cnt + TC_QTR - 1) / TC_QTR;  // quarters holding positions
      if (tid == 0) {
        // both buffers are free once every earlier bulk store has read them out
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        if (P.res)
          for (int q = 0; q < 2 && q < nq; ++q) {
            qtr_load(P, rbar + 8 * q, s_base + q * TC_SQ_BYTES, q0, cnt, q);
            ++rissued[q];
          }
      }
      ok = epi_all(mbar_wait(bar0 + 8 * (2 + acc), (i >> 1) & 1));
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int q = 0; q < nq && ok; ++q) {
        const int buf = q & 1;
        const int rows = min(TC_QTR, cnt - q * TC_QTR);
        const int64_t qq = (int64_t)(q0 + q * TC_QTR);
        float* S = sS + buf * (TC_QTR * TC_M);
        if (P.res) {
          ok = epi_all(mbar_wait(rbar + 8 * buf, rphase[buf] & 1));
          if (!ok) break;
          ++rphase[buf];
          if (tid == 0 && q >= 1 && q + 1 < nq) {
            // the store of quarter q - 1 has read S[1 - buf] before the next rows land there
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            qtr_load(P, rbar + 8 * (1 - buf), s_base + (1 - buf) * TC_SQ_BYTES, q0, cnt, q + 1);
            ++rissued[1 - buf];
          }
        } else {
          // the store of quarter q - 2 has read S[buf] (the latest one may still be reading the other)
          if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          epi_sync();
        }
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * TC_N + q * TC_QTR + sub * 16), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        uint32_t drop = 0;  // bit k: masked out
        if (P.mask) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int r = sub * 16 + k;
            if (r < rows && !(P.mask[(qq + r) * TC_M + m] > 0.f)) drop |= 1u << k;
          }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int r = sub * 16 + k;
          if (r < rows) {
            float* sp = S + r * TC_M + m;
            float val = ((drop >> k) & 1u) ? 0.f : __uint_as_float(v[k]) + bm;
            if (P.res) val += *sp;
            *sp = val;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        epi_sync();
        if (tid == 0) {
          asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(P.out + qq * TC_M),
                       "r"(s_base + buf * TC_SQ_BYTES), "r"((uint32_t)rows * TC_M * 4)
                       : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
      }
      if (!ok) break;
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(bar0 + 8 * (4 + acc));  // accumulator free (TC_EPI arrivals)
    }
    if (!ok && tid == 0) {
      atomicOr(P.error, 1u);
      // after a wait that gave up, let residual copies still in flight land
      // (bounded waits) before the CTA's shared memory is released
      for (int b = 0; b < 2; ++b)
        for (; rphase[b] < rissued[b]; ++rphase[b]) mbar_wait(rbar + 8 * b, rphase[b] & 1);
    }
    // the output is written and S read out before the CTA ends
    if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS) : "memory");
}

struct DwArgs {
  const float* dY;  // [npos][M]
  const float* X;   // [npos][Kc]
  float* dW;        // [M][taps][Kc], accumulated
  int M, Kc, taps, relu_in, npos, seq_len, qchunk;
};

// dW[m][n] += sum_q dY[q][m] act(X[q + t - c][j]), n = t Kc + j; blockIdx.z picks
// a chunk of positions; partial tiles are added with atomics.
__global__ void __launch_bounds__(kThreads) k_conv_dw(DwArgs P) {
  __shared__ __align__(16) uint16_t As[BM][BK + kPadK];
  __shared__ __align__(16) uint16_t Bs[BN][BK + kPadK];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int q_begin = blockIdx.z * P.qchunk;
  const int q_end = min(P.npos, q_begin + P.qchunk);
  const int warp = threadIdx.x >> 5, wm = warp >> 1, wn = warp & 1;
  const int c = (P.taps - 1) / 2;
  const int N = P.taps * P.Kc;
  float acc[2][4][4] = {};
  for (int k0 = q_begin; k0 < q_end; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK / 2; e += kThreads) {
      const int mm = e / (BK / 2), kk = 2 * (e % (BK / 2));
      const int m = m0 + mm;
      float v0 = 0.f, v1 = 0.f;
      if (m < P.M) {
        if (k0 + kk < q_end) v0 = P.dY[(int64_t)(k0 + kk) * P.M + m];
        if (k0 + kk + 1 < q_end) v1 = P.dY[(int64_t)(k0 + kk + 1) * P.M + m];
      }
      *reinterpret_cast<uint32_t*>(&As[mm][kk]) = pack_bf16(v0, v1);
    }
    for (int e = threadIdx.x; e < BN * BK / 2; e += kThreads) {
      const int nn = e / (BK / 2), kk = 2 * (e % (BK / 2));
      const int n = n0 + nn;
      float v[2] = {0.f, 0.f};
      if (n < N) {
        const int t = n / P.Kc, j = n - t * P.Kc;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = k0 + kk + h;
          if (q < q_end) {
            const int seq = q / P.seq_len, l = q - seq * P.seq_len;
            const int l2 = l + t - c;
            if (l2 >= 0 && l2 < P.seq_len) {
              const float x = P.X[((int64_t)seq * P.seq_len + l2) * P.Kc + j];
              v[h] = P.relu_in ? fmaxf(x, 0.f) : x;
            }
          }
        }
      }
      *reinterpret_cast<uint32_t*>(&Bs[nn][kk]) = pack_bf16(v[0], v[1]);
    }
    __syncthreads();
    warp_mma(As, Bs, wm, wn, 0, acc);
    warp_mma(As, Bs, wm, wn, 16, acc);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int m = m0 + wm * 32 + i * 16 + g + (h >= 2 ? 8 : 0);
        const int n = n0 + wn * 32 + j * 8 + 2 * t + (h & 1);
        if (m < P.M && n < N) atomicAdd(&P.dW[(int64_t)m * N + n], acc[i][j][h]);
      }
}

// db[m] += sum_q dY[q][m]
__global__ void k_bias_grad(const float* __restrict__ dY, int npos, int M, float* __restrict__ db) {
  const int m = blockIdx.x;
  float s = 0.f;
  for (int q = threadIdx.x; q < npos; q += blockDim.x) s += dY[(int64_t)q * M + m];
  __shared__ float red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[m] += red[0];
}

// Sum of the mask weights, into acc[0] (acc zeroed before).
__global__ void k_mask_sum(const float* __restrict__ mask, int64_t npts, double* __restrict__ acc) {
  double local = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npts;
       i += (int64_t)gridDim.x * blockDim.x)
    local += (double)mask[i];
  __shared__ double red[256];
  red[threadIdx.x] = local;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(acc, red[0]);
}

// Masked MSE with weights w = mask[point] and norm = cout sum(w) (acc[0]):
// loss (acc[1]) = sum w (y - target)^2 / norm, dy = 2 w (y - target) / norm.
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ target,
                      const float* __restrict__ mask, int64_t npts, int cout,
                      float* __restrict__ dy, double* __restrict__ acc) {
  const double norm = acc[0] * (double)cout;
  const float inv_norm = norm > 0.0 ? (float)(1.0 / norm) : 0.f;
  double local = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npts * cout;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float w = mask[i / cout];
    const float d = y[i] - target[i];
    dy[i] = 2.f * w * d * inv_norm;
    local += (double)w * (double)d * (double)d;
  }
  __shared__ double red[256];
  red[threadIdx.x] = local;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(acc + 1, red[0] * (double)inv_norm);
}

// Adam step on the FP32 master weights, then their BF16 copies.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// BF16 copy of one layer's weights W[o][t][i] and of its per-tap transpose
// WT[i][t][o] (the operand of the input-gradient pass).
__global__ void k_weights_bf16(const float* __restrict__ W, int Co, int taps, int Ci,
                               __nv_bfloat16* __restrict__ Wb, __nv_bfloat16* __restrict__ WTb) {
  const int64_t n = (int64_t)Co * taps * Ci;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int o = (int)(e / ((int64_t)taps * Ci));
    const int t = (int)((e / Ci) % taps);
    const int i = (int)(e % Ci);
    const __nv_bfloat16 b = __float2bfloat16_rn(W[e]);
    Wb[e] = b;
    if (WTb) WTb[((int64_t)i * taps + t) * Co + o] = b;
  }
}

}  // namespace

// ---------------------------------------------------------------------------

struct rpk_net {
  int cin = 0, cout = 0, width = 0, nblocks = 0, device = 0;
  cudaStream_t stream = nullptr;
  struct Layer {
    int Co, taps, Ci;
    int64_t w_off, b_off;      // offsets in the parameter vector
    int64_t wb_off;            // offset in the bf16 weight arrays
  };
  std::vector<Layer> layers;   // lift, (b0 c0, b0 c1, ...), head
  int64_t nparams = 0, nwb = 0;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *wb = nullptr, *wtb = nullptr;
  int64_t step = 0;
  // activation workspace for up to cap_q coarse positions
  int64_t cap_q = 0;
  float* act = nullptr;   // h_0..h_B (B+1), z0 per block (B): (2B+1) x cap_q x width
  float* work = nullptr;  // 2 x cap_q x width scratch for gradients
  float* headout = nullptr;
  float* dybuf = nullptr;
  double* loss = nullptr;
  int2* qseq = nullptr;        // ragged sequence table, cap_q entries
  int* starts = nullptr;       // ragged sequence starts, cap_seq + 1 entries
  int cap_seq = 0;
  int4* tiles = nullptr;       // ragged tensor-core tiles (q0, count, start, length)
  int ntiles = 0, cap_tiles = 0;
  unsigned* tc_error = nullptr;  // set by k_conv_tc when a wait gives up
  int nsm = 0;
  bool tc = false;             // the tensor-core path serves the block convolutions
};

namespace {

rpk_status net_alloc(void** p, size_t bytes) {
  cudaError_t err = cudaMalloc(p, bytes);
  if (err != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return rpk::fail(RPK_ERR_OOM, std::string("network allocation failed: ") + cudaGetErrorString(err));
  }
  return RPK_OK;
}

rpk_status ensure_workspace(rpk_net* N, int64_t nq) {
  if (nq <= N->cap_q) return RPK_OK;
  cudaFree(N->act);
  cudaFree(N->work);
  cudaFree(N->headout);
  cudaFree(N->dybuf);
  cudaFree(N->qseq);
  N->act = N->work = N->headout = N->dybuf = nullptr;
  N->qseq = nullptr;
  N->cap_q = 0;
  const size_t W = N->width;
  rpk_status st = net_alloc((void**)&N->act, sizeof(float) * (2 * N->nblocks + 1) * nq * W);
  if (st == RPK_OK) st = net_alloc((void**)&N->work, sizeof(float) * 2 * nq * W);
  if (st == RPK_OK) st = net_alloc((void**)&N->headout, sizeof(float) * nq * R * N->cout);
  if (st == RPK_OK) st = net_alloc((void**)&N->dybuf, sizeof(float) * nq * R * N->cout);
  if (st == RPK_OK) st = net_alloc((void**)&N->qseq, sizeof(int2) * nq);
  if (st != RPK_OK) return st;
  N->cap_q = nq;
  return RPK_OK;
}

// Error word of the tensor-core path (synchronises the stream).
rpk_status tc_status(rpk_net* N) {
  if (!N->tc_error) return RPK_OK;
  unsigned e = 0;
  RPK_CUDA(cudaMemcpyAsync(&e, N->tc_error, sizeof(unsigned), cudaMemcpyDeviceToHost, N->stream));
  RPK_CUDA(cudaStreamSynchronize(N->stream));
  if (e) return rpk::fail(RPK_ERR_CUDA, "tensor-core convolution: an mbarrier wait gave up");
  return RPK_OK;
}

rpk_status refresh_bf16(rpk_net* N) {
  for (const auto& L : N->layers) {
    const int64_t n = (int64_t)L.Co * L.taps * L.Ci;
    const int blocks = (int)std::min<int64_t>(1024, (n + 255) / 256);
    k_weights_bf16<<<blocks, 256, 0, N->stream>>>(N->w + L.w_off, L.Co, L.taps, L.Ci,
                                                   N->wb + L.wb_off, N->wtb + L.wb_off);
  }
  RPK_CUDA(cudaGetLastError());
  return RPK_OK;
}

rpk_status conv(rpk_net* N, const __nv_bfloat16* A, int M, int taps, int Kc, int sgn,
                const float* X, int relu_in, float* out, const float* bias, const float* res,
                const float* mask, int64_t nq, int seq_len, const int2* qseq = nullptr) {
  // 16-byte operands: the weights and inputs for cp.async, the output and
  // residual rows for the epilogue's bulk copies
  const bool aligned = (((uintptr_t)A | (uintptr_t)X | (uintptr_t)out | (uintptr_t)res) & 15) == 0;
  if (N->tc && M == TC_M && Kc == TC_KC && taps == TC_TAPS && aligned && nq > 0) {
    TcArgs T{A, X, out, bias, res, mask, nullptr, 0, seq_len, 0, sgn, relu_in, N->tc_error};
    if (qseq) {
      T.tiles = N->tiles;
      T.ntiles = N->ntiles;
    } else {
      T.tiles_per_seq = (seq_len + TC_N - 1) / TC_N;
      T.ntiles = (int)(nq / seq_len) * T.tiles_per_seq;
    }
    const int grid = std::max(1, std::min(T.ntiles, N->nsm));
    k_conv_tc<<<grid, TC_THREADS, TC_SMEM, N->stream>>>(T);
    RPK_CUDA(cudaGetLastError());
    return RPK_OK;
  }
  ConvArgs P{A, X, out, bias, res, mask, qseq, M, Kc, taps, sgn, relu_in, (int)nq, seq_len};
  const dim3 grid((unsigned)((nq + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
  k_conv<<<grid, kThreads, 0, N->stream>>>(P);
  RPK_CUDA(cudaGetLastError());
  return RPK_OK;
}

rpk_status conv_dw(rpk_net* N, const float* dY, int M, const float* X, int Kc, int taps,
                   int relu_in, float* dW, int64_t nq, int seq_len) {
  // positions per block: enough blocks for about four per SM over the
  // (output x input) tiles, between 128 and 2048 positions, a multiple of BK
  const int64_t tiles = (int64_t)((taps * Kc + BN - 1) / BN) * ((M + BM - 1) / BM);
  const int64_t want = std::max<int64_t>(1, 4 * (int64_t)std::max(N->nsm, 1) / std::max<int64_t>(tiles, 1));
  int64_t qc = (nq + want - 1) / want;
  qc = std::min<int64_t>(2048, std::max<int64_t>(128, (qc + BK - 1) / BK * BK));
  const int qchunk = (int)qc;
  DwArgs P{dY, X, dW, M, Kc, taps, relu_in, (int)nq, seq_len, qchunk};
  const dim3 grid((unsigned)((taps * Kc + BN - 1) / BN), (unsigned)((M + BM - 1) / BM),
                  (unsigned)((nq + qchunk - 1) / qchunk));
  k_conv_dw<<<grid, kThreads, 0, N->stream>>>(P);
  RPK_CUDA(cudaGetLastError());
  return RPK_OK;
}

// Forward pass over nq coarse positions (sequences of Lq positions each, or the
// sequences described by qseq); keeps the activations.
rpk_status forward(rpk_net* N, const float* x, int64_t nq, int Lq, const int2* qseq, float* y) {
  rpk_status st = ensure_workspace(N, nq);
  if (st != RPK_OK) return st;
  const int64_t stride = nq * N->width;
  float* h = N->act;  // h_b at act + b * stride; z0_b at act + (B + 1 + b) * stride
  const auto& lift = N->layers[0];
  st = conv(N, N->wb + lift.wb_off, N->width, 1, R * N->cin, +1, x, 0, h, N->w + lift.b_off,
            nullptr, nullptr, nq, Lq, qseq);
  for (int b = 0; b < N->nblocks && st == RPK_OK; ++b) {
    const auto& c0 = N->layers[1 + 2 * b];
    const auto& c1 = N->layers[2 + 2 * b];
    float* hb = N->act + b * stride;
    float* z0 = N->act + (N->nblocks + 1 + b) * stride;
    float* hn = N->act + (b + 1) * stride;
    st = conv(N, N->wb + c0.wb_off, N->width, K5, N->width, +1, hb, 1, z0, N->w + c0.b_off,
              nullptr, nullptr, nq, Lq, qseq);
    if (st == RPK_OK)
      st = conv(N, N->wb + c1.wb_off, N->width, K5, N->width, +1, z0, 1, hn, N->w + c1.b_off, hb,
                nullptr, nq, Lq, qseq);
  }
  if (st != RPK_OK) return st;
  const auto& head = N->layers.back();
  return conv(N, N->wb + head.wb_off, R * N->cout, 1, N->width, +1, N->act + N->nblocks * stride,
              1, y, N->w + head.b_off, nullptr, nullptr, nq, Lq, qseq);
}

// qseq[q] = (first position, length) of the sequence holding coarse position q;
// one block per sequence, starts[s] .. starts[s + 1] (coarse positions).
__global__ void k_fill_qseq(const int* __restrict__ starts, int2* __restrict__ qseq) {
  const int lo = starts[blockIdx.x], hi = starts[blockIdx.x + 1];
  for (int q = lo + threadIdx.x; q < hi; q += blockDim.x) qseq[q] = make_int2(lo, hi - lo);
}

// Backward pass from dy (fine layout == coarse layout), gradients into N->g.
rpk_status backward(rpk_net* N, const float* x, const float* dy, int nseq, int L) {
  const int64_t nq = (int64_t)nseq * (L / R);
  const int Lq = L / R;
  const int64_t stride = nq * N->width;
  RPK_CUDA(cudaMemsetAsync(N->g, 0, sizeof(float) * N->nparams, N->stream));
  float* dh = N->work;           // gradient wrt h (current block output)
  float* tmp = N->work + stride;  // gradient wrt z0
  const int W = N->width;
  const auto& head = N->layers.back();
  const float* hB = N->act + N->nblocks * stride;
  rpk_status st = conv_dw(N, dy, R * N->cout, hB, W, 1, 1, N->g + head.w_off, nq, Lq);
  k_bias_grad<<<R * N->cout, 256, 0, N->stream>>>(dy, (int)nq, R * N->cout, N->g + head.b_off);
  // d relu(h_B) = W_head^T dy, then mask by h_B > 0
  if (st == RPK_OK)
    st = conv(N, N->wtb + head.wb_off, W, 1, R * N->cout, -1, dy, 0, dh, nullptr, nullptr, hB, nq, Lq);
  for (int b = N->nblocks - 1; b >= 0 && st == RPK_OK; --b) {
    const auto& c0 = N->layers[1 + 2 * b];
    const auto& c1 = N->layers[2 + 2 * b];
    const float* hb = N->act + b * stride;
    const float* z0 = N->act + (N->nblocks + 1 + b) * stride;
    // z1 = conv(relu(z0)); d z1 = dh
    st = conv_dw(N, dh, W, z0, W, K5, 1, N->g + c1.w_off, nq, Lq);
    k_bias_grad<<<W, 256, 0, N->stream>>>(dh, (int)nq, W, N->g + c1.b_off);
    if (st == RPK_OK)
      st = conv(N, N->wtb + c1.wb_off, W, K5, W, -1, dh, 0, tmp, nullptr, nullptr, z0, nq, Lq);
    // z0 = conv(relu(h_b)); d z0 = tmp
    if (st == RPK_OK) st = conv_dw(N, tmp, W, hb, W, K5, 1, N->g + c0.w_off, nq, Lq);
    k_bias_grad<<<W, 256, 0, N->stream>>>(tmp, (int)nq, W, N->g + c0.b_off);
    // d h_b = dh + (W0^T tmp) masked by h_b > 0   (written in place of dh)
    if (st == RPK_OK)
      st = conv(N, N->wtb + c0.wb_off, W, K5, W, -1, tmp, 0, dh, nullptr, dh, hb, nq, Lq);
  }
  if (st != RPK_OK) return st;
  const auto& lift = N->layers[0];
  st = conv_dw(N, dh, W, x, R * N->cin, 1, 0, N->g + lift.w_off, nq, Lq);
  k_bias_grad<<<W, 256, 0, N->stream>>>(dh, (int)nq, W, N->g + lift.b_off);
  RPK_CUDA(cudaGetLastError());
  return st;
}

}  // namespace

extern "C" {

rpk_status rpk_net_create(int cin, int cout, int width, int nblocks, uint64_t seed,
                          void* cuda_stream, rpk_net** out) {
  if (!out) return rpk::fail(RPK_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (cin < 1 || cout < 1 || width < 16 || width % 16 || nblocks < 0 || nblocks > 64)
    return rpk::fail(RPK_ERR_ARG, "cin, cout >= 1; width a multiple of 16; 0 <= nblocks <= 64");
  rpk_net* N = new (std::nothrow) rpk_net();
  if (!N) return rpk::fail(RPK_ERR_OOM, "host allocation failed");
  N->cin = cin;
  N->cout = cout;
  N->width = width;
  N->nblocks = nblocks;
  N->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&N->device);
  auto add = [&](int Co, int taps, int Ci) {
    rpk_net::Layer L{Co, taps, Ci, N->nparams, N->nparams + (int64_t)Co * taps * Ci, N->nwb};
    N->nparams += (int64_t)Co * taps * Ci + Co;
    N->nwb += (int64_t)Co * taps * Ci;
    N->layers.push_back(L);
  };
  add(width, 1, R * cin);
  for (int b = 0; b < nblocks; ++b) {
    add(width, K5, width);
    add(width, K5, width);
  }
  add(R * cout, 1, width);
  // He-style initialisation drawn on the host; biases zero
  std::vector<float> w(N->nparams, 0.f);
  std::mt19937_64 rng(seed);
  for (size_t li = 0; li < N->layers.size(); ++li) {
    const auto& L = N->layers[li];
    const bool head = li + 1 == N->layers.size();
    const double sd = std::sqrt((head ? 1.0 : 2.0) / (L.taps * L.Ci));
    std::normal_distribution<double> nd(0.0, sd);
    for (int64_t i = 0; i < (int64_t)L.Co * L.taps * L.Ci; ++i) w[L.w_off + i] = (float)nd(rng);
  }
  rpk_status st = net_alloc((void**)&N->w, sizeof(float) * N->nparams);
  if (st == RPK_OK) st = net_alloc((void**)&N->g, sizeof(float) * N->nparams);
  if (st == RPK_OK) st = net_alloc((void**)&N->m, sizeof(float) * N->nparams);
  if (st == RPK_OK) st = net_alloc((void**)&N->v, sizeof(float) * N->nparams);
  if (st == RPK_OK) st = net_alloc((void**)&N->wb, sizeof(__nv_bfloat16) * N->nwb);
  if (st == RPK_OK) st = net_alloc((void**)&N->wtb, sizeof(__nv_bfloat16) * N->nwb);
  if (st == RPK_OK) st = net_alloc((void**)&N->loss, 2 * sizeof(double));
  if (st == RPK_OK) st = net_alloc((void**)&N->tc_error, sizeof(unsigned));
  if (st == RPK_OK) {
    cudaDeviceGetAttribute(&N->nsm, cudaDevAttrMultiProcessorCount, N->device);
    N->tc = width == TC_M &&
            cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM) ==
                cudaSuccess;
    cudaGetLastError();
  }
  cudaError_t err = cudaSuccess;
  if (st == RPK_OK)
    err = cudaMemcpyAsync(N->w, w.data(), sizeof(float) * N->nparams, cudaMemcpyHostToDevice, N->stream);
  if (st == RPK_OK && err == cudaSuccess) err = cudaMemsetAsync(N->m, 0, sizeof(float) * N->nparams, N->stream);
  if (st == RPK_OK && err == cudaSuccess) err = cudaMemsetAsync(N->v, 0, sizeof(float) * N->nparams, N->stream);
  if (st == RPK_OK && err == cudaSuccess) err = cudaMemsetAsync(N->tc_error, 0, sizeof(unsigned), N->stream);
  if (st == RPK_OK && err == cudaSuccess) st = refresh_bf16(N);
  if (st == RPK_OK && err == cudaSuccess) err = cudaStreamSynchronize(N->stream);
  if (st != RPK_OK || err != cudaSuccess) {
    if (st == RPK_OK) st = rpk::cuda_fail(err, "rpk_net_create");
    rpk_net_destroy(N);
    return st;
  }
  *out = N;
  return RPK_OK;
}

void rpk_net_destroy(rpk_net* N) {
  if (!N) return;
  cudaStreamSynchronize(N->stream);
  void* p[] = {N->w,    N->g,       N->m,     N->v,    N->wb,     N->wtb,  N->act,
               N->work, N->headout, N->dybuf, N->loss, N->qseq, N->starts, N->tiles, N->tc_error};
  for (void* q : p)
    if (q) cudaFree(q);
  delete N;
}

int64_t rpk_net_num_params(const rpk_net* N) { return N ? N->nparams : 0; }

rpk_status rpk_net_get_params(rpk_net* N, float* host, int which) {
  if (!N || !host) return rpk::fail(RPK_ERR_ARG, "NULL argument");
  const float* src = which == 1 ? N->g : N->w;
  RPK_CUDA(cudaMemcpyAsync(host, src, sizeof(float) * N->nparams, cudaMemcpyDeviceToHost, N->stream));
  RPK_CUDA(cudaStreamSynchronize(N->stream));
  return RPK_OK;
}

rpk_status rpk_net_set_params(rpk_net* N, const float* host) {
  if (!N || !host) return rpk::fail(RPK_ERR_ARG, "NULL argument");
  RPK_CUDA(cudaMemcpyAsync(N->w, host, sizeof(float) * N->nparams, cudaMemcpyHostToDevice, N->stream));
  rpk_status st = refresh_bf16(N);
  if (st != RPK_OK) return st;
  RPK_CUDA(cudaStreamSynchronize(N->stream));
  return RPK_OK;
}

rpk_status rpk_net_forward(rpk_net* N, const float* x, int nseq, int len, float* y) {
  if (!N || !x || !y) return rpk::fail(RPK_ERR_ARG, "NULL argument");
  if (nseq < 1 || len < R || len % R) return rpk::fail(RPK_ERR_ARG, "len must be a positive multiple of 4");
  RPK_CUDA(cudaSetDevice(N->device));
  return forward(N, x, (int64_t)nseq * (len / R), len / R, nullptr, y);
}

rpk_status rpk_net_forward_ragged(rpk_net* N, const float* x, int nseq, const int* lens, float* y) {
  if (!N || !x || !y || !lens) return rpk::fail(RPK_ERR_ARG, "NULL argument");
  if (nseq < 1) return rpk::fail(RPK_ERR_ARG, "nseq must be >= 1");
  std::vector<int> starts(nseq + 1, 0);
  for (int s = 0; s < nseq; ++s) {
    if (lens[s] < R || lens[s] % R)
      return rpk::fail(RPK_ERR_ARG, "every length must be a positive multiple of 4");
    if ((int64_t)starts[s] + lens[s] / R > INT32_MAX / 2)
      return rpk::fail(RPK_ERR_ARG, "too many positions");
    starts[s + 1] = starts[s] + lens[s] / R;
  }
  RPK_CUDA(cudaSetDevice(N->device));
  const int64_t nq = starts[nseq];
  rpk_status st = ensure_workspace(N, nq);
  if (st != RPK_OK) return st;
  if (nseq > N->cap_seq) {
    cudaFree(N->starts);
    N->starts = nullptr;
    N->cap_seq = 0;
    st = net_alloc((void**)&N->starts, sizeof(int) * (nseq + 1));
    if (st != RPK_OK) return st;
    N->cap_seq = nseq;
  }
  RPK_CUDA(cudaMemcpyAsync(N->starts, starts.data(), sizeof(int) * (nseq + 1),
                           cudaMemcpyHostToDevice, N->stream));
  // tensor-core tiles: 128 positions of one sequence each
  std::vector<int4> tiles;
  for (int s = 0; s < nseq; ++s)
    for (int q = starts[s]; q < starts[s + 1]; q += TC_N)
      tiles.push_back(make_int4(q, std::min(TC_N, starts[s + 1] - q), starts[s], starts[s + 1] - starts[s]));
  if ((int)tiles.size() > N->cap_tiles) {
    cudaFree(N->tiles);
    N->tiles = nullptr;
    N->cap_tiles = 0;
    st = net_alloc((void**)&N->tiles, sizeof(int4) * tiles.size());
    if (st != RPK_OK) return st;
    N->cap_tiles = (int)tiles.size();
  }
  N->ntiles = (int)tiles.size();
  RPK_CUDA(cudaMemcpyAsync(N->tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice,
                           N->stream));
  k_fill_qseq<<<nseq, 256, 0, N->stream>>>(N->starts, N->qseq);
  RPK_CUDA(cudaGetLastError());
  st = forward(N, x, nq, 0, N->qseq, y);
  // the host tables are read before they go away
  if (st == RPK_OK) RPK_CUDA(cudaStreamSynchronize(N->stream));
  if (st == RPK_OK) st = tc_status(N);
  return st;
}

rpk_status rpk_net_loss_grad(rpk_net* N, const float* x, const float* target, const float* mask,
                             int nseq, int len, double* loss) {
  if (!N || !x || !target || !mask || !loss) return rpk::fail(RPK_ERR_ARG, "NULL argument");
  if (nseq < 1 || len < R || len % R) return rpk::fail(RPK_ERR_ARG, "len must be a positive multiple of 4");
  RPK_CUDA(cudaSetDevice(N->device));
  const int64_t nq = (int64_t)nseq * (len / R);
  rpk_status st = ensure_workspace(N, nq);
  if (st != RPK_OK) return st;
  float* y = N->headout;
  st = forward(N, x, nq, len / R, nullptr, y);
  if (st != RPK_OK) return st;
  RPK_CUDA(cudaMemsetAsync(N->loss, 0, 2 * sizeof(double), N->stream));
  const int64_t npts = (int64_t)nseq * len;
  k_mask_sum<<<256, 256, 0, N->stream>>>(mask, npts, N->loss);
  k_mse<<<512, 256, 0, N->stream>>>(y, target, mask, npts, N->cout, N->dybuf, N->loss);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) st = backward(N, x, N->dybuf, nseq, len);
  if (err == cudaSuccess && st == RPK_OK)
    err = cudaMemcpyAsync(loss, N->loss + 1, sizeof(double), cudaMemcpyDeviceToHost, N->stream);
  if (err == cudaSuccess && st == RPK_OK) err = cudaStreamSynchronize(N->stream);
  if (st != RPK_OK) return st;
  if (err != cudaSuccess) return rpk::cuda_fail(err, "rpk_net_loss_grad");
  return tc_status(N);
}

rpk_status rpk_net_adam(rpk_net* N, float lr, float beta1, float beta2, float eps) {
  if (!N) return rpk::fail(RPK_ERR_ARG, "NULL network");
  RPK_CUDA(cudaSetDevice(N->device));
  N->step += 1;
  const float c1 = 1.f - (float)std::pow((double)beta1, (double)N->step);
  const float c2 = 1.f - (float)std::pow((double)beta2, (double)N->step);
  k_adam<<<1024, 256, 0, N->stream>>>(N->w, N->g, N->m, N->v, N->nparams, lr, beta1, beta2, eps, c1, c2);
  RPK_CUDA(cudaGetLastError());
  return refresh_bf16(N);
}

}  // extern "C"
