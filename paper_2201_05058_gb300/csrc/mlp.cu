// BF16 multilayer perceptron with FP32 accumulation on sm_103a tensor cores:
// the learned surrogate of the dynamic (human) distance field.
//
// Network: 16 inputs (11 features, 5 zero pads) -> 256 -> 256 -> 256 -> 1, ReLU
// after the three hidden layers.  Weights live as FP32 master copies (Adam) and
// BF16 copies (GEMM operands); activations and back-propagated gradients are
// stored in BF16, every product is accumulated in FP32.
//
// Kernels:
//   k_gemm     C(m,n) = sum_k A(m,k) B(k,n) with mma.sync m16n8k16 (BF16 in, FP32
//              accumulate), operands staged in shared memory; the epilogue
//              adds the bias and applies ReLU (forward), multiplies by the
//              ReLU mask of the layer below (input gradient) or accumulates
//              FP32 into a weight gradient (split over the batch).
//   k_head     the 256 -> 1 output layer, the squared-error loss and its
//              gradient with respect to the last hidden layer.
//   k_colsum   bias gradients (column sums of a BF16 gradient matrix).
//   k_adam     Adam update of the FP32 master copy and refresh of the BF16 copy.
//   k_init     counter-hash uniform initialisation (fan-in scaled).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "host.h"

using namespace pcdf::host;

namespace pcdf {
namespace mlp {

constexpr int kW = PCDF_MLP_WIDTH;   // 256
constexpr int kIn = PCDF_MLP_IN_PAD; // 16

// element offsets of the FP32 parameter vector
constexpr long long oW1 = 0, oB1 = oW1 + (long long)kW * kIn, oW2 = oB1 + kW, oB2 = oW2 + (long long)kW * kW,
                    oW3 = oB2 + kW, oB3 = oW3 + (long long)kW * kW, oW4 = oB3 + kW, oB4 = oW4 + kW,
                    kP = oB4 + 1, kPpad = (kP + 3) / 4 * 4;
// element offsets of the BF16 weight copies
constexpr long long hW1 = 0, hW2 = hW1 + (long long)kW * kIn, hW3 = hW2 + (long long)kW * kW,
                    hW4 = hW3 + (long long)kW * kW, kH = hW4 + kW;
static_assert(kP == PCDF_MLP_PARAMS, "parameter count");
static_assert(kH == PCDF_MLP_BF16_WEIGHTS, "bf16 weight count");

// state layout (bytes): master, adam m, adam v, grad (FP32 [kPpad] each), bf16 weights
// then the hidden BF16 weights again, packed for the tensor-core kernel
constexpr size_t sMaster = 0, sM = 4 * kPpad, sV = 8 * kPpad, sGrad = 12 * kPpad, sHalf = 16 * kPpad,
                 sPack = (sHalf + 2 * kH + 255) / 256 * 256, kPackElems = 2LL * kW * kW,
                 kStateBytes = sPack + 2 * kPackElems;

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------------------
// GEMM
// ---------------------------------------------------------------------------
constexpr int BM = 64, BN = 64, BK = 32, PADK = 8;

enum Epi { kBiasRelu = 0, kMask = 1, kAtomic = 2 };

struct GemmArgs {
    const bf16 *A, *B;
    int lda, ldb, M, N, K, k_split;
    const float *bias;   // kBiasRelu
    const bf16 *mask;    // kMask: output zero where mask <= 0
    int ldm;
    bf16 *out_h;         // kBiasRelu, kMask
    float *out_f;        // kAtomic
    int ldo;
};

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Stage a 64 x BK tile whose element (r, k) is at P[r * ld + k] (kT = false)
// or P[k * ld + r] (kT = true) into S[r][k]; out-of-range elements are zero.
template <bool kT>
__device__ __forceinline__ void stage_tile(bf16 (*S)[BK + PADK], const bf16 *__restrict__ P, int ld, int r0, int R,
                                           int k0, int k1)
{
    const bf16 zero = __float2bfloat16_rn(0.f);
    for (int v = threadIdx.x; v < BM * BK / 8; v += blockDim.x) {
        if (!kT) {
            const int r = v / (BK / 8), kq = (v % (BK / 8)) * 8;
            const int gr = r0 + r, gk = k0 + kq;
            if (gr < R && gk + 8 <= k1) {
                const uint4 q = *reinterpret_cast<const uint4 *>(P + (long long)gr * ld + gk);
                *reinterpret_cast<uint4 *>(&S[r][kq]) = q;
            } else {
                for (int j = 0; j < 8; ++j)
                    S[r][kq + j] = (gr < R && gk + j < k1) ? P[(long long)gr * ld + gk + j] : zero;
            }
        } else {
            const int k = v / (BM / 8), rq = (v % (BM / 8)) * 8;
            const int gk = k0 + k, gr = r0 + rq;
            if (gk < k1 && gr + 8 <= R) {
                const uint4 q = *reinterpret_cast<const uint4 *>(P + (long long)gk * ld + gr);
                const bf16 *e = reinterpret_cast<const bf16 *>(&q);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    S[rq + j][k] = e[j];
            } else {
                for (int j = 0; j < 8; ++j)
                    S[rq + j][k] = (gk < k1 && gr + j < R) ? P[(long long)gk * ld + gr + j] : zero;
            }
        }
    }
}

template <bool kTA, bool kTB, int kEpi>
__global__ void __launch_bounds__(128) k_gemm(const GemmArgs g)
{
    __shared__ __align__(16) bf16 As[BM][BK + PADK];
    __shared__ __align__(16) bf16 Bs[BN][BK + PADK];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * g.k_split, ke = min(g.K, kb + g.k_split);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp >> 1, wn = warp & 1, gid = lane >> 2, tig = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                acc[i][j][q] = 0.f;

    for (int k0 = kb; k0 < ke; k0 += BK) {
        stage_tile<kTA>(As, g.A, g.lda, m0, g.M, k0, ke);
        stage_tile<kTB>(Bs, g.B, g.ldb, n0, g.N, k0, ke);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r = wm * 32 + mt * 16 + gid, c = kk + tig * 2;
                a[mt][0] = *reinterpret_cast<const uint32_t *>(&As[r][c]);
                a[mt][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][c]);
                a[mt][2] = *reinterpret_cast<const uint32_t *>(&As[r][c + 8]);
                a[mt][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][c + 8]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int n = wn * 32 + nt * 8 + gid, k = kk + tig * 2;
                b[nt][0] = *reinterpret_cast<const uint32_t *>(&Bs[n][k]);
                b[nt][1] = *reinterpret_cast<const uint32_t *>(&Bs[n][k + 8]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
                    mma16816(acc[mt][nt], a[mt], b[nt]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = m0 + wm * 32 + mt * 16 + gid + (q >= 2 ? 8 : 0);
                const int c = n0 + wn * 32 + nt * 8 + tig * 2 + (q & 1);
                if (r >= g.M || c >= g.N)
                    continue;
                const float v = acc[mt][nt][q];
                if (kEpi == kBiasRelu) {
                    g.out_h[(long long)r * g.ldo + c] = __float2bfloat16_rn(fmaxf(v + g.bias[c], 0.f));
                } else if (kEpi == kMask) {
                    const float m = __bfloat162float(g.mask[(long long)r * g.ldm + c]);
                    g.out_h[(long long)r * g.ldo + c] = __float2bfloat16_rn(m > 0.f ? v : 0.f);
                } else {
                    atomicAdd(g.out_f + (long long)r * g.ldo + c, v);
                }
            }
}

template <bool kTA, bool kTB, int kEpi>
cudaError_t gemm(const GemmArgs &g, int splits, cudaStream_t st)
{
    const dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, splits);
    k_gemm<kTA, kTB, kEpi><<<grid, 128, 0, st>>>(g);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fused inference: the whole network for a tile of rows in one CTA
// ---------------------------------------------------------------------------
// The activations of the tile stay in shared memory between layers; the
// hidden weights stream through a double-buffered shared-memory chunk
// (cp.async).  Per output element the k16 products are accumulated in the
// same order as k_gemm and the epilogues and head do the same arithmetic as
// k_gemm's bias+ReLU and k_head, so y is bit-identical to forward + head.
constexpr int kIR = 64;           // rows per CTA
constexpr int kIT = 256;          // threads: 8 warps, 2 (rows) x 4 (columns)
constexpr int kKC = 32;           // K chunk of a hidden weight matrix
constexpr int kActLd = kW + 8;    // row strides in bf16 (padding against bank conflicts)
constexpr int kWLd = kKC + 8;
constexpr int kInLd = kIn + 8;
constexpr int kChunks = 2 * (kW / kKC);  // W2 then W3
constexpr size_t kInferSmem =
    ((size_t)kIR * kActLd + 2 * (size_t)kW * kWLd + (size_t)kIR * kInLd + (size_t)kW * kInLd) * sizeof(bf16);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

// 16-byte async copy; src_bytes 0 writes zeros
__device__ __forceinline__ void cp16(void *dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// one k16 step of the warp's 32 x 64 block: A rows from `a` (row stride lda,
// columns k0 ..), B = W rows n (stride ldb, columns kb ..)
__device__ __forceinline__ void warp_k16(float (&acc)[2][8][4], const bf16 *a, int lda, int k0, const bf16 *w,
                                         int ldb, int kb, int wm, int wn, int lane)
{
    uint32_t af[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
        ldsm_x4(af[mt], a + (wm * 32 + mt * 16 + (lane & 15)) * lda + k0 + (lane >> 4) * 8);
#pragma unroll
    for (int np = 0; np < 4; ++np) {
        uint32_t r[4];
        ldsm_x4(r, w + (wn * 64 + np * 16 + (lane & 7) + ((lane >> 4) << 3)) * ldb + kb + ((lane >> 3) & 1) * 8);
        const uint32_t b0[2] = {r[0], r[1]}, b1[2] = {r[2], r[3]};
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            mma16816(acc[mt][2 * np], af[mt], b0);
            mma16816(acc[mt][2 * np + 1], af[mt], b1);
        }
    }
}

// act[r][c] = bf16(max(acc + bias[c], 0)) for the warp's block
__device__ __forceinline__ void warp_epilogue(bf16 *act, const float (&acc)[2][8][4], const float *__restrict__ bias,
                                              int wm, int wn, int lane)
{
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int hq = 0; hq < 2; ++hq) {
                const int r = wm * 32 + mt * 16 + gid + 8 * hq;
                const int c = wn * 64 + nt * 8 + tig * 2;
                __nv_bfloat162 v;
                v.x = __float2bfloat16_rn(fmaxf(acc[mt][nt][2 * hq] + __ldg(bias + c), 0.f));
                v.y = __float2bfloat16_rn(fmaxf(acc[mt][nt][2 * hq + 1] + __ldg(bias + c + 1), 0.f));
                *reinterpret_cast<__nv_bfloat162 *>(act + r * kActLd + c) = v;
            }
}

__global__ void __launch_bounds__(kIT, 2) k_mlp_infer(const bf16 *__restrict__ wh, const float *__restrict__ p,
                                                      const bf16 *__restrict__ x, long long M, float *__restrict__ y)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 *act = reinterpret_cast<bf16 *>(smem_raw);
    bf16 *wbuf = act + kIR * kActLd;       // [2][kW][kWLd]
    bf16 *xs = wbuf + 2 * kW * kWLd;       // [kIR][kInLd]
    bf16 *w1s = xs + kIR * kInLd;          // [kW][kInLd]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, wm = warp >> 2, wn = warp & 3;
    const long long m0 = (long long)blockIdx.x * kIR;
    const bf16 *W1 = wh + hW1, *W2 = wh + hW2, *W3 = wh + hW3;

    // x tile (rows past M read as zeros) and W1: 16-byte pieces
    for (int v = tid; v < kIR * 2; v += kIT) {
        const int r = v >> 1, h = (v & 1) * 8;
        const bool in = m0 + r < M;
        cp16(xs + r * kInLd + h, x + (in ? (m0 + r) * kIn + h : 0), in ? 16 : 0);
    }
    for (int v = tid; v < kW * 2; v += kIT) {
        const int n = v >> 1, h = (v & 1) * 8;
        cp16(w1s + n * kInLd + h, W1 + n * kIn + h, 16);
    }
    cp_commit();
    auto issue = [&](int g) {  // chunk g: W2 (g < 8) or W3, columns kKC * (g % 8) ..
        const bf16 *W = g < kW / kKC ? W2 : W3;
        const int kb = (g % (kW / kKC)) * kKC;
        bf16 *dst = wbuf + (g & 1) * kW * kWLd;
        for (int v = tid; v < kW * (kKC / 8); v += kIT) {
            const int n = v / (kKC / 8), q = (v % (kKC / 8)) * 8;
            cp16(dst + n * kWLd + q, W + n * kW + kb + q, 16);
        }
        cp_commit();
    };
    issue(0);

    float acc[2][8][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                acc[mt][nt][q] = 0.f;
    cp_wait_all();
    __syncthreads();
    // layer 1 (K = 16: one k16 step)
    warp_k16(acc, xs, kInLd, 0, w1s, kInLd, 0, wm, wn, lane);
    warp_epilogue(act, acc, p + oB1, wm, wn, lane);

    // layers 2 and 3
    for (int g = 0; g < kChunks; ++g) {
        if (g % (kW / kKC) == 0) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        acc[mt][nt][q] = 0.f;
        }
        cp_wait_all();     // this thread's pieces of chunk g have landed
        __syncthreads();   // everyone's have; chunk g - 1 and the layer input are done with
        if (g + 1 < kChunks)
            issue(g + 1);
        const bf16 *wc = wbuf + (g & 1) * kW * kWLd;
        const int k0 = (g % (kW / kKC)) * kKC;
#pragma unroll
        for (int kk = 0; kk < kKC; kk += 16)
            warp_k16(acc, act, kActLd, k0 + kk, wc, kWLd, kk, wm, wn, lane);
        if (g % (kW / kKC) == kW / kKC - 1) {
            __syncthreads();  // every warp has read the layer input
            warp_epilogue(act, acc, p + (g < kW / kKC ? oB2 : oB3), wm, wn, lane);
        }
    }
    __syncthreads();

    // head: the 256 -> 1 layer, as k_head (lane j owns columns 8 j .. 8 j + 7)
    float w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        w[j] = __bfloat162float(wh[hW4 + lane * 8 + j]);
    const float b4 = p[oB4];
    for (int i = warp; i < kIR; i += kIT / 32) {
        const long long m = m0 + i;
        if (m >= M)
            break;
        const uint4 q = *reinterpret_cast<const uint4 *>(act + i * kActLd + lane * 8);
        const bf16 *hh = reinterpret_cast<const bf16 *>(&q);
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            s = fmaf(__bfloat162float(hh[j]), w[j], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0)
            y[m] = s + b4;
    }
}

// ---------------------------------------------------------------------------
// fused inference on the 5th-generation tensor cores (tcgen05 + TMEM)
// ---------------------------------------------------------------------------
// Each layer of a 128-row tile is D[128 x 256] = A[128 x K] B[256 x K]^T with
// D in tensor memory (256 fp32 columns, row r in lane r): one thread issues
// tcgen05.mma (kind::f16, BF16 operands in shared memory, FP32 accumulate)
// and commits to mbarriers; the epilogue warps read the accumulator back with
// tcgen05.ld, add the bias, apply ReLU and store the BF16 activations as the
// next layer's A operand.  The head reads the last layer from tensor memory.
//
// W2 and W3 are pre-packed (k_pack_hidden) into 8 chunks of 64 columns, each
// laid out exactly as the B operand in shared memory, so one bulk copy moves
// a chunk.
//
// Operand tiles use the canonical K-major layout without swizzling: 8 x 16
// byte core matrices (8 rows of 8 BF16); element (r, k) of a tile with Kt
// columns is at byte (r / 8) * Kt * 16 + (k / 8) * 128 + (r % 8) * 16 +
// (k % 8) * 2, so K-adjacent core matrices are 128 bytes apart (leading byte
// offset) and 8-row groups Kt * 16 bytes apart (stride byte offset).
//
// Every mbarrier wait gives up after about a second: the CTA then writes NaN
// for its remaining rows, gives the operations it issued a second bounded
// wait, and frees its tensor memory on every path.
namespace tc {

constexpr int kM = 128, kKC = 64;  // tile rows; K columns of a packed weight chunk
constexpr uint64_t kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t kmaj(int r, int k, int Kt)
{
    return (uint32_t)((r >> 3) * Kt * 16 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start, leading and stride byte offsets (all
// >> 4), the fixed 0b001 at bits 46-48, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B BF16 (bits
// 7-9 and 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kW >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// 32 consecutive fp32 columns of the calling thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i)
        v[i] = __uint_as_float(r[i]);
}

// the same load without its wait: r may be read only after tmem_wait_ld(r),
// which takes the registers as in-out operands so that no use moves above it
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count = 1)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// one arrival expecting `bytes` of copy completions, then the bulk copy
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try(bar, parity))
        return true;
    const uint64_t t0 = now_ns();
    while (!mbar_try(bar, parity))
        if (now_ns() - t0 > kWaitNs)
            return false;
    return true;
}

}  // namespace tc

// W2 and W3 into the chunked B-operand layout: chunk j (layer j / 4, columns
// 64 (j % 4) ..) holds element (n, k) at tc::kmaj(n, k, 64) / 2
__global__ void k_pack_hidden(const bf16 *__restrict__ wh, bf16 *__restrict__ packed)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;  // one 16-byte piece
    if (v >= 2 * kW * (kW / 8))
        return;
    const int l = v / (kW * (kW / 8)), rem = v % (kW * (kW / 8));
    const int n = rem / (kW / 8), kq = rem % (kW / 8);
    const bf16 *W = wh + (l == 0 ? hW2 : hW3);
    const int k = kq * 8, chunk = l * (kW / tc::kKC) + k / tc::kKC;
    bf16 *dst = packed + (long long)chunk * (kW * tc::kKC) + tc::kmaj(n, k % tc::kKC, tc::kKC) / 2;
    *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(W + n * kW + k);
}

// ---------------------------------------------------------------------------
// The kernel is persistent and warp-specialised: one CTA per SM walks its
// 128-row tiles with three roles working concurrently on mbarriers
//   warp 0 (one thread)  issues the products and commits;
//   warp 1               producer: the x tiles (double-buffered) and the
//                        packed W2/W3 chunks through the 4-stage ring;
//   warps 2..9           epilogue: warp w reads TMEM lanes 32 (w % 4) .. and,
//                        in group g = (w - 2) / 4, the 32-column slices
//                        g, g + 2, g + 4, g + 6 of every layer.
// Tensor memory holds two 256-column accumulators; the layers of the CTA's
// tiles (q = 3 * tile + layer) alternate between them, so the epilogue of
// layer q overlaps the products of layer q + 1: the four products of chunk c
// (64 columns) of layer q + 1 are issued as soon as the two groups holding its
// slices have written those columns of its A operand (barrier aready[c]), and
// an accumulator is overwritten only after every epilogue thread has read it
// (accempty).  The head sums each group's
// columns and the groups are added in a fixed order.
// ---------------------------------------------------------------------------
namespace ws {
constexpr int kStages = 4, kEpiWarps = 8, kGroups = kEpiWarps / 4, kThreads = 32 * (2 + kEpiWarps);
constexpr int kSlices = 8 / kGroups;  // 32-column slices of a layer per epilogue warp
constexpr int kChunks = kW / tc::kKC;  // chunks of a hidden layer
constexpr uint32_t kCols = 512;
constexpr uint32_t kBytesA = 128 * kW * 2, kBytesChunk = kW * tc::kKC * 2, kBytesX = 128 * kIn * 2,
                   kBytesW1 = kW * kIn * 2;
constexpr uint32_t oA = 0, oRing = oA + kBytesA, oX = oRing + kStages * kBytesChunk, oW1 = oX + 2 * kBytesX,
                   oBias = oW1 + kBytesW1, oW4 = oBias + 3 * kW * 4, oPart = oW4 + kW * 4,
                   kEnd = oPart + 2 * kGroups * 128 * 4;
constexpr size_t kSmem = 1024 + (size_t)kEnd;
static_assert(kSmem <= 227 * 1024, "shared memory");
static_assert(kEpiWarps % 4 == 0 && 8 % kGroups == 0 && kGroups % 2 == 0,
              "groups of four warps; the two slices of a 64-column chunk belong to two groups");

// lane 0's value for every lane of the (converged) warp, through the warp's
// own shared slot, so that the warp takes every branch as a whole
__device__ __forceinline__ int warp_uniform(int v, volatile int *slot, int lane)
{
    if (lane == 0)
        *slot = v;
    __syncwarp();
    const int u = *slot;
    __syncwarp();
    return u;
}
// a bounded wait taken by lane 0 on behalf of the warp
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *slot, int lane)
{
    return warp_uniform(lane == 0 ? (int)tc::mbar_wait(bar, parity) : 0, slot, lane) != 0;
}
}  // namespace ws

// relu of two floats rounded to BF16 (nearest even), low half first, in one
// conversion (rounding keeps the sign, so relu before or after it agree)
__device__ __forceinline__ uint32_t bf2_relu_bits(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
// relu(v + b) of a pair rounded to BF16 as above, the two additions in one
// paired FP32 instruction (each lane an IEEE round-to-nearest add)
__device__ __forceinline__ uint32_t bf2_bias_relu_bits(float v0, float v1, float b0, float b1)
{
    uint32_t d;
    asm("{\n\t.reg .b64 a, b, s;\n\t.reg .f32 lo, hi;\n\t"
        "mov.b64 a, {%1, %2};\n\tmov.b64 b, {%3, %4};\n\tadd.rn.f32x2 s, a, b;\n\t"
        "mov.b64 {lo, hi}, s;\n\tcvt.rn.relu.bf16x2.f32 %0, hi, lo;\n\t}"
        : "=r"(d)
        : "f"(v0), "f"(v1), "f"(b0), "f"(b1));
    return d;
}
// (a0, a1) += (x0, x1) * (y0, y1), each lane an IEEE fused multiply-add
__device__ __forceinline__ void fma2(float &a0, float &a1, float x0, float x1, float y0, float y1)
{
    asm("{\n\t.reg .b64 a, x, y;\n\t"
        "mov.b64 a, {%0, %1};\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\t"
        "fma.rn.f32x2 a, x, y, a;\n\tmov.b64 {%0, %1}, a;\n\t}"
        : "+f"(a0), "+f"(a1)
        : "f"(x0), "f"(x1), "f"(y0), "f"(y1));
}

__global__ void __launch_bounds__(ws::kThreads, 1)
    k_mlp_infer_ws(const bf16 *__restrict__ wh, const float *__restrict__ p, const bf16 *__restrict__ packed,
                   const bf16 *__restrict__ x, long long M, const int32_t *__restrict__ count, float *__restrict__ y)
{
    // rows: M, or the first *count of them when a device count is given
    if (count) {
        const long long c = *count;
        M = c < 0 ? 0 : (c < M ? c : M);
    }
    const long long ntiles = (M + 127) / 128;
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t full[ws::kStages], empty[ws::kStages], xfull[2], xempty[2], accfull[2], accempty[2],
        aready[ws::kChunks], partfull[2], drain;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_fail;
    __shared__ volatile int s_slot[2 + ws::kEpiWarps];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    unsigned char *sA = base + ws::oA, *sRing = base + ws::oRing, *sX = base + ws::oX, *sW1 = base + ws::oW1;
    float *sBias = reinterpret_cast<float *>(base + ws::oBias), *sW4 = reinterpret_cast<float *>(base + ws::oW4),
          *sPart = reinterpret_cast<float *>(base + ws::oPart);
    const uint32_t aA = smem_u32(sA), aRing = smem_u32(sRing), aX = smem_u32(sX), aW1 = smem_u32(sW1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0)
        tc::tmem_alloc(&s_tmem, ws::kCols);
    if (tid == 0) {
        for (int i = 0; i < ws::kStages; ++i) {
            tc::mbar_init(&full[i]);
            tc::mbar_init(&empty[i]);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&xfull[i], 32);
            tc::mbar_init(&xempty[i]);
            tc::mbar_init(&accfull[i]);
            tc::mbar_init(&accempty[i], ws::kEpiWarps * 32);
            tc::mbar_init(&partfull[i], ws::kEpiWarps * 32);
        }
        for (int j = 0; j < ws::kChunks; ++j)
            tc::mbar_init(&aready[j], 2 * 4 * 32);  // two slices, each written by the four warps of its group
        tc::mbar_init(&drain);
        tc::fence_mbar_init();
        s_fail = 0;
    }
    // W1, the biases and the head weights.  The first layer's bias rides in
    // the product: the x tiles carry 1 in their three padding columns (13,
    // 14, 15) and W1 gets b1 there, split into three BF16 parts whose sum is
    // b1 to FP32 rounding (high part, then the high parts of the remainders).
    static_assert(kIn == 16 && PCDF_MLP_IN == 13, "three padding columns carry the first bias");
    for (int v = tid; v < kW * 2; v += ws::kThreads) {
        const int n = v >> 1, h = (v & 1) * 8;
        uint4 w = __ldg(reinterpret_cast<const uint4 *>(wh + hW1 + n * kIn + h));
        if (h == 8) {
            const float b = p[oB1 + n];
            const __nv_bfloat16 bh = __float2bfloat16_rn(b);
            const float r1 = b - __bfloat162float(bh);
            const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
            const __nv_bfloat16 bl = __float2bfloat16_rn(r1 - __bfloat162float(bm));
            // elements 8..15 of the row: k = 13 is the high half of .z, 14 and 15 are .w
            w.z = (w.z & 0xFFFFu) | ((uint32_t)__bfloat16_as_ushort(bh) << 16);
            w.w = (uint32_t)__bfloat16_as_ushort(bm) | ((uint32_t)__bfloat16_as_ushort(bl) << 16);
        }
        *reinterpret_cast<uint4 *>(sW1 + tc::kmaj(n, h, kIn)) = w;
    }
    for (int i = tid; i < kW; i += ws::kThreads) {
        sBias[i] = p[oB1 + i];
        sBias[kW + i] = p[oB2 + i];
        sBias[2 * kW + i] = p[oB3 + i];
        sW4[i] = __bfloat162float(wh[hW4 + i]);
    }
    cp_commit();
    cp_wait_all();
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    const float b4 = p[oB4];

    if (warp == 0) {
        // ---- products -----------------------------------------------------
        if (lane == 0) {
            long long g = 0;  // chunks consumed
            bool ok = true;
            int it = 0;
            for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
                const int b = it & 1;
                const long long q1 = 3LL * it;
                ok = tc::mbar_wait(&xfull[b], (uint32_t)(it >> 1) & 1u) &&
                     (q1 < 2 || tc::mbar_wait(&accempty[q1 & 1], (uint32_t)((q1 - 2) >> 1) & 1u));
                if (!ok)
                    break;
                tc::fence_after();
                tc::mma(tmem + (uint32_t)(q1 & 1) * 256u, tc::sdesc(aX + b * ws::kBytesX, 128, kIn * 16),
                        tc::sdesc(aW1, 128, kIn * 16), 0u);
                tc::commit(&xempty[b]);
                tc::commit(&accfull[q1 & 1]);
                for (int L = 1; L <= 2 && ok; ++L) {
                    const long long q = q1 + L;
                    const uint32_t dcol = tmem + (uint32_t)(q & 1) * 256u;
                    if (q >= 2 && !tc::mbar_wait(&accempty[q & 1], (uint32_t)((q - 2) >> 1) & 1u)) {
                        ok = false;
                        break;
                    }
                    const uint32_t aph = (uint32_t)(2 * it + L - 1) & 1u;
                    for (int c = 0; c < ws::kChunks; ++c, ++g) {
                        const int st = (int)(g % ws::kStages);
                        if (!tc::mbar_wait(&full[st], (uint32_t)(g / ws::kStages) & 1u) ||
                            !tc::mbar_wait(&aready[c], aph)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after();
#pragma unroll
                        for (int kk = 0; kk < tc::kKC / 16; ++kk) {
                            const int k0 = tc::kKC * c + 16 * kk;
                            tc::mma(dcol, tc::sdesc(aA + (uint32_t)(k0 / 8) * 128u, 128, kW * 16),
                                    tc::sdesc(aRing + (uint32_t)(st * ws::kBytesChunk + kk * 256), 128, tc::kKC * 16),
                                    (uint32_t)(c | kk));
                        }
                        tc::commit(&empty[st]);
                    }
                    if (ok)
                        tc::commit(&accfull[q & 1]);
                }
                if (s_fail)
                    ok = false;
            }
            if (!ok)
                s_fail = 1;
            // every product issued has finished before the tensor memory is freed
            tc::commit(&drain);
            (void)tc::mbar_wait(&drain, 0);
        }
    } else if (warp == 1) {
        // ---- producer -----------------------------------------------------
        volatile int *slot = s_slot + 1;
        long long g = 0;  // chunks issued (lane 0)
        int it = 0;
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int b = it & 1;
            int stop = 0;
            if (lane == 0) {
                stop = s_fail;
                if (!stop && it >= 2 && !tc::mbar_wait(&xempty[b], (uint32_t)((it >> 1) - 1) & 1u))
                    stop = s_fail = 1;
            }
            if (ws::warp_uniform(stop, slot, lane))
                break;
            const long long m0 = tile * 128;
            unsigned char *xb = sX + b * ws::kBytesX;
#pragma unroll
            for (int v = lane; v < 256; v += 32) {
                const int r = v >> 1, h = (v & 1) * 8;
                uint4 val = make_uint4(0u, 0u, 0u, 0u);
                if (m0 + r < M)
                    val = __ldg(reinterpret_cast<const uint4 *>(x + (m0 + r) * kIn + h));
                if (h == 8) {  // the padding columns 13, 14, 15 carry 1 (the first bias, above)
                    val.z = (val.z & 0xFFFFu) | (0x3F80u << 16);
                    val.w = 0x3F803F80u;
                }
                *reinterpret_cast<uint4 *>(xb + tc::kmaj(r, h, kIn)) = val;
            }
            tc::fence_proxy_async();
            tc::mbar_arrive(&xfull[b]);
            if (lane == 0) {
                for (int c = 0; c < 2 * ws::kChunks; ++c, ++g) {
                    const int st = (int)(g % ws::kStages);
                    if (g >= ws::kStages && !tc::mbar_wait(&empty[st], (uint32_t)(g / ws::kStages - 1) & 1u)) {
                        s_fail = 1;
                        break;
                    }
                    tc::bulk_load(sRing + st * ws::kBytesChunk, packed + (long long)c * (kW * tc::kKC),
                                  ws::kBytesChunk, &full[st]);
                }
            }
        }
        if (lane == 0) {
            // copies still in flight are among the last kStages issued
            for (long long c = g > ws::kStages ? g - ws::kStages : 0; c < g; ++c)
                (void)tc::mbar_wait(&full[c % ws::kStages], (uint32_t)(c / ws::kStages) & 1u);
        }
    } else {
        // ---- epilogue -----------------------------------------------------
        const int quarter = warp & 3, group = (warp - 2) >> 2;
        const int r = quarter * 32 + lane;
        volatile int *slot = s_slot + warp;
        long long pend = -1;  // tile whose head sums wait to be added (group 0)
        int pend_it = 0;
        auto flush_pending = [&]() -> bool {
            if (!ws::warp_wait(&partfull[pend_it & 1], (uint32_t)(pend_it >> 1) & 1u, slot, lane))
                return false;
            const float *part = sPart + (pend_it & 1) * (ws::kGroups * 128);
            float sum = 0.f;
#pragma unroll
            for (int g2 = 0; g2 < ws::kGroups; ++g2)
                sum += part[g2 * 128 + r];
            if (pend * 128 + r < M)
                y[pend * 128 + r] = sum + b4;
            pend = -1;
            return true;
        };
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        // this warp's slices group, group + kGroups, ... of the accumulator at
        // tb; the next slice's load is in flight while f converts the current
        auto each_slice = [&](uint32_t tb, auto &&f) {
            uint32_t va[32], vb[32];
            tc::tmem_ld32_async(tb + (uint32_t)(32 * group), va);
            tc::tmem_wait_ld(va);
#pragma unroll
            for (int k = 0; k < ws::kSlices; ++k) {
                const int j = group + k * ws::kGroups;
                uint32_t(&cur)[32] = (k & 1) ? vb : va;
                uint32_t(&nxt)[32] = (k & 1) ? va : vb;
                if (k + 1 < ws::kSlices)
                    tc::tmem_ld32_async(tb + (uint32_t)(32 * (j + ws::kGroups)), nxt);
                f(cur, j);
                if (k + 1 < ws::kSlices)
                    tc::tmem_wait_ld(nxt);
            }
        };
        int it = 0;
        long long tile = blockIdx.x;
        bool ok = true;
        for (; tile < ntiles; tile += gridDim.x, ++it) {
            for (int L = 0; L < 3 && ok; ++L) {
                const long long q = 3LL * it + L;
                const int a = (int)(q & 1);
                if (!ws::warp_wait(&accfull[a], (uint32_t)(q >> 1) & 1u, slot, lane)) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                const uint32_t tb = tmem + (uint32_t)a * 256u + lane_off;
                if (L < 2) {
                    const float *bias = sBias + L * kW;
                    const bool with_bias = L == 1;  // the first layer's bias came with its product
                    // slice j (32 columns): bias, ReLU, BF16 into the A operand, then
                    // its chunk's barrier; the next slice's load is in flight meanwhile
                    auto slice = [&](const uint32_t(&v)[32], int j) {
#pragma unroll
                        for (int gq = 0; gq < 4; ++gq) {
                            const uint32_t *u = v + 8 * gq;
                            uint4 pk;
                            if (with_bias) {
                                const float4 b0 = *reinterpret_cast<const float4 *>(bias + 32 * j + 8 * gq);
                                const float4 b1 = *reinterpret_cast<const float4 *>(bias + 32 * j + 8 * gq + 4);
                                pk.x = bf2_bias_relu_bits(__uint_as_float(u[0]), __uint_as_float(u[1]), b0.x, b0.y);
                                pk.y = bf2_bias_relu_bits(__uint_as_float(u[2]), __uint_as_float(u[3]), b0.z, b0.w);
                                pk.z = bf2_bias_relu_bits(__uint_as_float(u[4]), __uint_as_float(u[5]), b1.x, b1.y);
                                pk.w = bf2_bias_relu_bits(__uint_as_float(u[6]), __uint_as_float(u[7]), b1.z, b1.w);
                            } else {
                                pk.x = bf2_relu_bits(__uint_as_float(u[0]), __uint_as_float(u[1]));
                                pk.y = bf2_relu_bits(__uint_as_float(u[2]), __uint_as_float(u[3]));
                                pk.z = bf2_relu_bits(__uint_as_float(u[4]), __uint_as_float(u[5]));
                                pk.w = bf2_relu_bits(__uint_as_float(u[6]), __uint_as_float(u[7]));
                            }
                            *reinterpret_cast<uint4 *>(sA + tc::kmaj(r, 32 * j + 8 * gq, kW)) = pk;
                        }
                        tc::fence_proxy_async();
                        tc::fence_before();
                        tc::mbar_arrive(&aready[j >> 1]);
                    };
                    each_slice(tb, slice);
                    tc::mbar_arrive(&accempty[a]);
                } else {
                    // head: relu(D + b3) rounded to BF16 (as stored between layers), . w4,
                    // in four partial sums
                    float acc4[4] = {0.f, 0.f, 0.f, 0.f};
                    auto slice = [&](const uint32_t(&v)[32], int j) {
#pragma unroll
                        for (int gq = 0; gq < 8; ++gq) {
                            const float4 b = *reinterpret_cast<const float4 *>(sBias + 2 * kW + 32 * j + 4 * gq);
                            const float4 w = *reinterpret_cast<const float4 *>(sW4 + 32 * j + 4 * gq);
                            const uint32_t *u = v + 4 * gq;
                            const uint32_t p0 = bf2_bias_relu_bits(__uint_as_float(u[0]), __uint_as_float(u[1]), b.x, b.y);
                            const uint32_t p1 = bf2_bias_relu_bits(__uint_as_float(u[2]), __uint_as_float(u[3]), b.z, b.w);
                            fma2(acc4[0], acc4[1], __uint_as_float(p0 << 16), __uint_as_float(p0 & 0xffff0000u), w.x,
                                 w.y);
                            fma2(acc4[2], acc4[3], __uint_as_float(p1 << 16), __uint_as_float(p1 & 0xffff0000u), w.z,
                                 w.w);
                        }
                    };
                    each_slice(tb, slice);
                    tc::fence_before();
                    tc::mbar_arrive(&accempty[a]);
                    sPart[(it & 1) * (ws::kGroups * 128) + group * 128 + r] = (acc4[0] + acc4[1]) + (acc4[2] + acc4[3]);
                    tc::mbar_arrive(&partfull[it & 1]);
                    // group 0 adds the groups' sums once it has written the next
                    // tile's first-layer activations (off the critical path)
                    pend = tile;
                    pend_it = it;
                }
                if (L == 0 && group == 0 && pend >= 0 && !flush_pending()) {
                    ok = false;
                    break;
                }
            }
            if (!ok || ws::warp_uniform(s_fail, slot, lane))
                break;
        }
        bool failed = !ok || ws::warp_uniform(s_fail, slot, lane);
        if (!failed && group == 0 && pend >= 0 && !flush_pending())
            failed = true;
        if (failed) {
            s_fail = 1;
            // the pending tile, this tile and the CTA's later ones have no answer
            if (group == 0) {
                if (pend >= 0 && pend * 128 + r < M)
                    y[pend * 128 + r] = __int_as_float(0x7fc00000);
                for (; tile < ntiles; tile += gridDim.x)
                    if (tile * 128 + r < M)
                        y[tile * 128 + r] = __int_as_float(0x7fc00000);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, ws::kCols);
    }
}

// ---------------------------------------------------------------------------
// output layer, loss, bias gradients, Adam, initialisation
// ---------------------------------------------------------------------------
constexpr int kHeadRows = 64;  // rows per CTA of k_head (8 warps x 8 rows)

// y[m] = H3[m] . w4 + b4.  With a target: loss += (y - t)^2 / M,
// dy = 2 (y - t) / M, dZ3[m][k] = dy * w4[k] where H3[m][k] > 0, and the
// gradients of w4 and b4 accumulate (per CTA in shared memory, then atomics).
__global__ void __launch_bounds__(256)
    k_head(const bf16 *__restrict__ H3, const bf16 *__restrict__ w4h, const float *__restrict__ b4, long long M,
           float *__restrict__ y, const float *__restrict__ target, bf16 *__restrict__ dZ3, float *__restrict__ gw4,
           float *__restrict__ gb4, float *__restrict__ loss, float inv_m)
{
    __shared__ float s_gw[kW];
    __shared__ float s_gb, s_loss;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < kW; k += blockDim.x)
        s_gw[k] = 0.f;
    if (threadIdx.x == 0)
        s_gb = s_loss = 0.f;
    __syncthreads();
    float w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        w[j] = __bfloat162float(w4h[lane * 8 + j]);
    float gw[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    float gb = 0.f, ls = 0.f;
    for (int i = warp; i < kHeadRows; i += blockDim.x / 32) {
        const long long m = (long long)blockIdx.x * kHeadRows + i;
        if (m >= M)
            break;
        const uint4 q = *reinterpret_cast<const uint4 *>(H3 + m * kW + lane * 8);
        const bf16 *h = reinterpret_cast<const bf16 *>(&q);
        float hv[8], s = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            hv[j] = __bfloat162float(h[j]);
            s = fmaf(hv[j], w[j], s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, o);
        const float yv = s + b4[0];
        if (lane == 0)
            y[m] = yv;
        if (target) {
            const float e = yv - target[m];
            const float dy = 2.f * e * inv_m;
            ls += e * e * inv_m;
            gb += dy;
            bf16 dz[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                dz[j] = __float2bfloat16_rn(hv[j] > 0.f ? dy * w[j] : 0.f);
                gw[j] = fmaf(dy, hv[j], gw[j]);
            }
            *reinterpret_cast<uint4 *>(dZ3 + m * kW + lane * 8) = *reinterpret_cast<const uint4 *>(dz);
        }
    }
    if (target) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            atomicAdd(&s_gw[lane * 8 + j], gw[j]);
        if (lane == 0) {
            atomicAdd(&s_gb, gb);
            atomicAdd(&s_loss, ls);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kW; k += blockDim.x)
            atomicAdd(gw4 + k, s_gw[k]);
        if (threadIdx.x == 0) {
            atomicAdd(gb4, s_gb);
            if (loss)
                atomicAdd(loss, s_loss);
        }
    }
}

// grad_b[n] += sum_m dZ[m][n] over a block of rows
__global__ void __launch_bounds__(256) k_colsum(const bf16 *__restrict__ dZ, long long M, float *__restrict__ gb)
{
    const int n = threadIdx.x;  // blockDim = kW
    const long long m0 = (long long)blockIdx.x * 256, m1 = min(M, m0 + 256);
    float s = 0.f;
    for (long long m = m0; m < m1; ++m)
        s += __bfloat162float(dZ[m * kW + n]);
    atomicAdd(gb + n, s);
}

__device__ __forceinline__ long long half_index(long long i)
{
    if (i < oB1)
        return hW1 + (i - oW1);
    if (i >= oW2 && i < oB2)
        return hW2 + (i - oW2);
    if (i >= oW3 && i < oB3)
        return hW3 + (i - oW3);
    if (i >= oW4 && i < oB4)
        return hW4 + (i - oW4);
    return -1;
}

__global__ void k_adam(float *__restrict__ p, float *__restrict__ mo, float *__restrict__ ve,
                       const float *__restrict__ g, bf16 *__restrict__ h, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kP)
        return;
    // input columns 11..15 of the first layer stay zero
    if (i < oB1 && (i % kIn) >= PCDF_MLP_IN)
        return;
    const float gi = g[i];
    const float m = b1 * mo[i] + (1.f - b1) * gi;
    const float v = b2 * ve[i] + (1.f - b2) * gi * gi;
    mo[i] = m;
    ve[i] = v;
    const float pn = p[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    p[i] = pn;
    const long long hi = half_index(i);
    if (hi >= 0)
        h[hi] = __float2bfloat16_rn(pn);
}

__device__ __forceinline__ uint32_t hash32(uint64_t x)
{
    // splitmix64 finaliser
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (uint32_t)(x >> 32);
}

// weights uniform in +-sqrt(6 / fan_in) (fan-in of the real inputs), biases 0,
// Adam moments 0
__global__ void k_init(float *__restrict__ p, float *__restrict__ mo, float *__restrict__ ve, bf16 *__restrict__ h,
                       unsigned long long seed)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kP)
        return;
    float fan = 0.f;
    if (i < oB1)
        fan = (i % kIn) < PCDF_MLP_IN ? (float)PCDF_MLP_IN : 0.f;
    else if ((i >= oW2 && i < oB2) || (i >= oW3 && i < oB3) || (i >= oW4 && i < oB4))
        fan = (float)kW;
    float v = 0.f;
    if (fan > 0.f) {
        const float u = (hash32(seed * 0x100000001B3ull + (unsigned long long)i) + 0.5f) * (1.f / 4294967296.f);
        v = (2.f * u - 1.f) * sqrtf(6.f / fan);
    }
    p[i] = v;
    mo[i] = 0.f;
    ve[i] = 0.f;
    const long long hi = half_index(i);
    if (hi >= 0)
        h[hi] = __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct State {
    float *p, *m, *v, *g;
    bf16 *h, *pk;  // BF16 weights; W2 and W3 packed for the tensor-core kernel
    explicit State(void *s)
    {
        char *b = (char *)s;
        p = (float *)(b + sMaster);
        m = (float *)(b + sM);
        v = (float *)(b + sV);
        g = (float *)(b + sGrad);
        h = (bf16 *)(b + sHalf);
        pk = (bf16 *)(b + sPack);
    }
};

// refreshes the packed copy of W2 and W3 after the BF16 weights change
__global__ void k_pack_hidden(const bf16 *__restrict__ wh, bf16 *__restrict__ packed);
cudaError_t launch_pack(const State &S, cudaStream_t st)
{
    k_pack_hidden<<<(2 * kW * (kW / 8) + 255) / 256, 256, 0, st>>>(S.h, S.pk);
    return cudaGetLastError();
}

// Workspace sections (each 256-byte aligned, in this order): the stored
// activations H1, H2, H3 and the stored pre-activation gradients D3, D2, D1
// (BF16 [M][256] each); see pcdf_mlp_backward.
struct Acts {
    bf16 *H1, *H2, *H3, *D3, *D2, *D1;
};

size_t ws_bytes(long long M) { return 6 * align_up((size_t)M * kW * 2); }

Acts carve(void *ws, long long M)
{
    char *b = (char *)ws;
    const size_t a = align_up((size_t)M * kW * 2);
    Acts r;
    r.H1 = (bf16 *)b;
    r.H2 = (bf16 *)(b + a);
    r.H3 = (bf16 *)(b + 2 * a);
    r.D3 = (bf16 *)(b + 3 * a);
    r.D2 = (bf16 *)(b + 4 * a);
    r.D1 = (bf16 *)(b + 5 * a);
    return r;
}

GemmArgs fwd_args(const bf16 *X, int K, const bf16 *W, const float *bias, bf16 *out, long long M)
{
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.A = X;
    g.lda = K;
    g.B = W;
    g.ldb = K;
    g.M = (int)M;
    g.N = kW;
    g.K = K;
    g.k_split = K;
    g.bias = bias;
    g.out_h = out;
    g.ldo = kW;
    return g;
}

int forward(const State &S, const bf16 *x, long long M, const Acts &A, cudaStream_t st)
{
    cudaError_t e = gemm<false, false, kBiasRelu>(fwd_args(x, kIn, S.h + hW1, S.p + oB1, A.H1, M), 1, st);
    if (e == cudaSuccess)
        e = gemm<false, false, kBiasRelu>(fwd_args(A.H1, kW, S.h + hW2, S.p + oB2, A.H2, M), 1, st);
    if (e == cudaSuccess)
        e = gemm<false, false, kBiasRelu>(fwd_args(A.H2, kW, S.h + hW3, S.p + oB3, A.H3, M), 1, st);
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "mlp forward");
}

// dX = dZ W with the ReLU mask of X (layer input); dZ [M][kW], W [kW][Kin]
cudaError_t back_input(const bf16 *dZ, const bf16 *W, int Kin, const bf16 *X, bf16 *dX, long long M, cudaStream_t st)
{
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.A = dZ;
    g.lda = kW;
    g.B = W;      // B(k = n_out, n = k_in) at W[k * Kin + n]
    g.ldb = Kin;
    g.M = (int)M;
    g.N = Kin;
    g.K = kW;
    g.k_split = kW;
    g.mask = X;
    g.ldm = Kin;
    g.out_h = dX;
    g.ldo = Kin;
    return gemm<false, true, kMask>(g, 1, st);
}

// gW[n][k] += sum_m dZ[m][n] X[m][k]
cudaError_t back_weight(const bf16 *dZ, const bf16 *X, int Kin, float *gW, long long M, cudaStream_t st)
{
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.A = dZ;     // A(m' = n, k' = m) at dZ[k' * kW + m']
    g.lda = kW;
    g.B = X;      // B(k' = m, n' = k) at X[k' * Kin + n']
    g.ldb = Kin;
    g.M = kW;
    g.N = Kin;
    g.K = (int)M;
    int splits = (int)std::min<long long>(128, (M + 2047) / 2048);
    splits = std::max(splits, 1);
    g.k_split = (int)(((M + splits - 1) / splits + BK - 1) / BK * BK);
    splits = (int)((M + g.k_split - 1) / g.k_split);
    g.out_f = gW;
    g.ldo = Kin;
    return gemm<true, true, kAtomic>(g, splits, st);
}

}  // namespace mlp
}  // namespace pcdf

using namespace pcdf::mlp;

namespace pcdf {
namespace mlp {
namespace {
int infer_tc(const void *state, const uint16_t *x, int64_t M, const int32_t *count, float *y, void *stream)
{
    if (!state || (M > 0 && (!x || !y)))
        return fail(PCDF_EINVAL, "state, x and y must be non-NULL");
    if (M < 0 || M > (1LL << 31) - 1)
        return fail(PCDF_EINVAL, "M out of range");
    if (M == 0)
        return PCDF_OK;
    if (!aligned(x, 16) || !aligned(state, kAlign))
        return fail(PCDF_EINVAL, "x must be 16-byte aligned, state %zu-byte aligned", kAlign);
    State S(const_cast<void *>(state));
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_infer_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws::kSmem);
    if (e == cudaSuccess) {
        // persistent: one CTA per SM (or per tile of the M rows, if fewer)
        const long long ntiles = (M + 127) / 128;
        k_mlp_infer_ws<<<(unsigned)(ntiles < nsm ? ntiles : nsm), ws::kThreads, ws::kSmem, st>>>(
            S.h, S.p, S.pk, (const bf16 *)x, M, count, y);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "mlp inference (tcgen05)");
}
}  // namespace
}  // namespace mlp
}  // namespace pcdf

extern "C" {

int pcdf_mlp_state_bytes(size_t *bytes)
{
    if (!bytes)
        return fail(PCDF_EINVAL, "bytes is NULL");
    *bytes = kStateBytes;
    return PCDF_OK;
}

int pcdf_mlp_workspace_bytes(int64_t M, size_t *bytes)
{
    if (!bytes || M < 0)
        return fail(PCDF_EINVAL, "bytes is NULL or M < 0");
    *bytes = ws_bytes(M);
    return PCDF_OK;
}

int pcdf_mlp_init(void *state, uint64_t seed, void *stream)
{
    if (!state || !aligned(state, kAlign))
        return fail(PCDF_EINVAL, "state must be non-NULL and %zu-byte aligned", kAlign);
    State S(state);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(S.g, 0, 4 * kPpad, st);
    if (e == cudaSuccess) {
        k_init<<<(unsigned)((kP + 255) / 256), 256, 0, st>>>(S.p, S.m, S.v, S.h, (unsigned long long)seed);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = launch_pack(S, st);
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "mlp init");
}

int pcdf_mlp_forward(const void *state, const uint16_t *x, int64_t M, float *y, void *workspace,
                     size_t workspace_bytes, void *stream)
{
    if (!state || (M > 0 && (!x || !y || !workspace)))
        return fail(PCDF_EINVAL, "state, x, y and workspace must be non-NULL");
    if (M < 0 || M > (1LL << 31) - 1)
        return fail(PCDF_EINVAL, "M out of range");
    if (M == 0)
        return PCDF_OK;
    if (!aligned(x, 16) || !aligned(workspace, kAlign) || !aligned(state, kAlign))
        return fail(PCDF_EINVAL, "x must be 16-byte aligned, state and workspace %zu-byte aligned", kAlign);
    if (workspace_bytes < ws_bytes(M))
        return fail(PCDF_ENOMEM, "workspace %zu bytes < %zu needed", workspace_bytes, ws_bytes(M));
    State S(const_cast<void *>(state));
    Acts A = carve(workspace, M);
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = forward(S, (const bf16 *)x, M, A, st))
        return rc;
    k_head<<<(unsigned)((M + kHeadRows - 1) / kHeadRows), 256, 0, st>>>(A.H3, S.h + hW4, S.p + oB4, M, y, nullptr,
                                                                        nullptr, nullptr, nullptr, nullptr, 0.f);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "mlp head");
}

int pcdf_mlp_infer(const void *state, const uint16_t *x, int64_t M, float *y, void *stream)
{
    if (!state || (M > 0 && (!x || !y)))
        return fail(PCDF_EINVAL, "state, x and y must be non-NULL");
    if (M < 0 || M > (1LL << 31) - 1)
        return fail(PCDF_EINVAL, "M out of range");
    if (M == 0)
        return PCDF_OK;
    if (!aligned(x, 16) || !aligned(state, kAlign))
        return fail(PCDF_EINVAL, "x must be 16-byte aligned, state %zu-byte aligned", kAlign);
    State S(const_cast<void *>(state));
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInferSmem);
    if (e == cudaSuccess) {
        k_mlp_infer<<<(unsigned)((M + kIR - 1) / kIR), kIT, kInferSmem, st>>>(S.h, S.p, (const bf16 *)x, M, y);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "mlp inference");
}


int pcdf_mlp_infer_tc(const void *state, const uint16_t *x, int64_t M, float *y, void *stream)
{
    return pcdf::mlp::infer_tc(state, x, M, nullptr, y, stream);
}

int pcdf_mlp_infer_tc_count(const void *state, const uint16_t *x, int64_t M_max, const int32_t *count, float *y,
                            void *stream)
{
    if (!count)
        return fail(PCDF_EINVAL, "count must be non-NULL");
    return pcdf::mlp::infer_tc(state, x, M_max, count, y, stream);
}

int pcdf_mlp_backward(void *state, const uint16_t *x, const float *target, int64_t M, float *y, float *loss,
                      void *workspace, size_t workspace_bytes, void *stream)
{
    if (!state || !x || !target || !y || !workspace)
        return fail(PCDF_EINVAL, "state, x, target, y and workspace must be non-NULL");
    if (M < 1 || M > (1LL << 31) - 1)
        return fail(PCDF_EINVAL, "M out of range");
    if (!aligned(x, 16) || !aligned(workspace, kAlign) || !aligned(state, kAlign))
        return fail(PCDF_EINVAL, "x must be 16-byte aligned, state and workspace %zu-byte aligned", kAlign);
    if (workspace_bytes < ws_bytes(M))
        return fail(PCDF_ENOMEM, "workspace %zu bytes < %zu needed", workspace_bytes, ws_bytes(M));
    State S(state);
    Acts A = carve(workspace, M);
    cudaStream_t st = (cudaStream_t)stream;
    const bf16 *X = (const bf16 *)x;
    cudaError_t e = cudaMemsetAsync(S.g, 0, 4 * kPpad, st);
    if (e == cudaSuccess && loss)
        e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess)
        return cuda_fail(e, "mlp backward reset");
    if (int rc = forward(S, X, M, A, st))
        return rc;
    k_head<<<(unsigned)((M + kHeadRows - 1) / kHeadRows), 256, 0, st>>>(A.H3, S.h + hW4, S.p + oB4, M, y, target,
                                                                        A.D3, S.g + oW4, S.g + oB4, loss,
                                                                        1.f / (float)M);
    e = cudaGetLastError();
    const unsigned cs = (unsigned)((M + 255) / 256);
    // layer 3: Z3 = H2 W3^T + b3
    if (e == cudaSuccess) {
        k_colsum<<<cs, kW, 0, st>>>(A.D3, M, S.g + oB3);
        e = back_weight(A.D3, A.H2, kW, S.g + oW3, M, st);
    }
    if (e == cudaSuccess)
        e = back_input(A.D3, S.h + hW3, kW, A.H2, A.D2, M, st);
    // layer 2
    if (e == cudaSuccess) {
        k_colsum<<<cs, kW, 0, st>>>(A.D2, M, S.g + oB2);
        e = back_weight(A.D2, A.H1, kW, S.g + oW2, M, st);
    }
    if (e == cudaSuccess)
        e = back_input(A.D2, S.h + hW2, kW, A.H1, A.D1, M, st);
    // layer 1 (the input needs no gradient)
    if (e == cudaSuccess) {
        k_colsum<<<cs, kW, 0, st>>>(A.D1, M, S.g + oB1);
        e = back_weight(A.D1, X, kIn, S.g + oW1, M, st);
    }
    if (e == cudaSuccess)
        e = cudaGetLastError();
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "mlp backward");
}

int pcdf_mlp_adam(void *state, float lr, float beta1, float beta2, float eps, int32_t step, void *stream)
{
    if (!state || step < 1)
        return fail(PCDF_EINVAL, "state must be non-NULL and step >= 1");
    State S(state);
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    cudaStream_t st = (cudaStream_t)stream;
    k_adam<<<(unsigned)((kP + 255) / 256), 256, 0, st>>>(S.p, S.m, S.v, S.g, S.h, lr, beta1, beta2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_pack(S, st);
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "mlp adam");
}

}  // extern "C"
