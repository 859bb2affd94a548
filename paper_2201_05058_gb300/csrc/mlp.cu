// BF16 multilayer perceptron with FP32 accumulation on sm_103a tensor cores:
// the learned surrogate of the dynamic (human) distance field.
//
// Network: 16 inputs (11 features, 5 zero pads) -> 256 -> 256 -> 256 -> 1, ReLU
// after the three hidden layers.  Weights live as FP32 master copies (Adam) and
// BF16 copies (GEMM operands); activations and back-propagated gradients are
// stored in BF16, every product is accumulated in FP32.
//
// Kernels:
//   k_mlp_ws<0>  inference: persistent, warp-specialised, tcgen05.mma with the
//                accumulators in tensor memory (all three layers and the head
//                of a 128-row tile without leaving the SM).
//   k_mlp_ws<1>  the same pass storing H1, H2, H3 for training or inspection.
//   k_mlp_ws<2>  the forward of a training step: H1, H2 stored, then the
//                head's backward (loss, dy, the w4 and b4 gradients).
//   k_mlp_dgrad  D3 = dy w4 masked by H3 > 0 (built on chip), D2 = (D3 W3)
//                masked by H2 > 0 and D1 = (D2 W2) masked by H1 > 0, tcgen05
//                with the packed transposed weights.
//   k_mlp_wgrad  the weight gradients D_l^T H_{l-1} (tcgen05, MN-major
//                operands, split over the batch) and the bias gradients.
//   k_mlp_infer  the legacy mma.sync m16n8k16 inference (baseline).
//   k_adam       Adam update of the FP32 master copy and refresh of the BF16 copy.
//   k_init       counter-hash uniform initialisation (fan-in scaled).
//   k_pack_hidden  the hidden weights (and their transposes) in the chunked
//                tensor-core operand layout.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
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
// then the hidden BF16 weights again, packed for the tensor-core kernels: W2,
// W3 (forward) and W3^T, W2^T (input gradients), in that order
constexpr size_t sMaster = 0, sM = 4 * kPpad, sV = 8 * kPpad, sGrad = 12 * kPpad, sHalf = 16 * kPpad,
                 sPack = (sHalf + 2 * kH + 255) / 256 * 256, kPackElems = 4LL * kW * kW,
                 kStateBytes = sPack + 2 * kPackElems;

using bf16 = __nv_bfloat16;

// mma.sync m16n8k16: BF16 in, FP32 accumulate (the legacy tensor-core path)
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ---------------------------------------------------------------------------
// fused inference: the whole network for a tile of rows in one CTA
// ---------------------------------------------------------------------------
// The legacy path (mma.sync, kept as the baseline of the tcgen05 kernels):
// the activations of the tile stay in shared memory between layers; the
// hidden weights stream through a double-buffered shared-memory chunk
// (cp.async).  Same arithmetic as the tcgen05 kernels up to the order of the
// FP32 sums.
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

    // head: the 256 -> 1 layer (lane j owns columns 8 j .. 8 j + 7)
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
// a chunk; W3^T and W2^T follow in 8 more chunks for the input gradients.
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

// the same for an M = 128 product of width n (a multiple of 16, up to 256);
// with mn_major both operands are MN-major (transposed, bits 15 and 16): then
// the leading byte offset of a descriptor is still the step between K-adjacent
// core matrices and the stride byte offset the step between MN-adjacent ones
__host__ __device__ constexpr uint32_t idesc(int n, bool mn_major)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (mn_major ? (1u << 15) | (1u << 16) : 0u) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}
static_assert(idesc(kW, false) == kIdesc, "instruction descriptor");

__device__ __forceinline__ void mma_i(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}

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
// one arrival expecting `bytes` of copy completions, for copies issued next
__device__ __forceinline__ void expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// a bulk copy that completes its bytes on `bar` (no arrival of its own)
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// bulk copy of shared memory to global memory in the calling thread's bulk
// group; wait_read returns once the source may be overwritten, wait_all once
// the writes are done
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
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

// W2, W3, W3^T and W2^T into the chunked B-operand layout: chunk j (matrix
// j / 4, K columns 64 (j % 4) ..) holds element (n, k) at tc::kmaj(n, k, 64) / 2,
// where element (n, k) is W[n][k] for W2 and W3 and W[k][n] for the transposes
// (n an input unit of the layer, k an output unit)
__global__ void k_pack_hidden(const bf16 *__restrict__ wh, bf16 *__restrict__ packed)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;  // one 16-byte piece
    if (v >= 4 * kW * (kW / 8))
        return;
    const int l = v / (kW * (kW / 8)), rem = v % (kW * (kW / 8));
    const int n = rem / (kW / 8), kq = rem % (kW / 8);
    const int k = kq * 8, chunk = l * (kW / tc::kKC) + k / tc::kKC;
    bf16 *dst = packed + (long long)chunk * (kW * tc::kKC) + tc::kmaj(n, k % tc::kKC, tc::kKC) / 2;
    if (l < 2) {
        const bf16 *W = wh + (l == 0 ? hW2 : hW3);
        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(W + n * kW + k);
    } else {
        const bf16 *W = wh + (l == 2 ? hW3 : hW2);
        __align__(16) bf16 e[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            e[i] = W[(k + i) * kW + n];
        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(e);
    }
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
                   oDY = oPart + 2 * kGroups * 128 * 4, kEnd = oDY + kBytesX;
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
// An epilogue warp's slices of the accumulator at tb (its lane quarter),
// for kG groups of four warps: the k-th is j = group + k kG; f(v, j, k) gets
// the 32 columns of slice j while the next slice's load is in flight.
template <int kG = kGroups, class F>
__device__ __forceinline__ void each_slice(uint32_t tb, int group, F &&f)
{
    constexpr int kS = 8 / kG;
    uint32_t va[32], vb[32];
    tc::tmem_ld32_async(tb + (uint32_t)(32 * group), va);
    tc::tmem_wait_ld(va);
#pragma unroll
    for (int k = 0; k < kS; ++k) {
        const int j = group + k * kG;
        uint32_t(&cur)[32] = (k & 1) ? vb : va;
        uint32_t(&nxt)[32] = (k & 1) ? va : vb;
        if (k + 1 < kS)
            tc::tmem_ld32_async(tb + (uint32_t)(32 * (j + kG)), nxt);
        f(cur, j, k);
        if (k + 1 < kS)
            tc::tmem_wait_ld(nxt);
    }
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

// Training outputs of the persistent kernel (modes 1 and 2).  Tiles of an
// [M][256] matrix are stored packed: element (m, k) at byte 65536 (m / 128) +
// tc::kmaj(m % 128, k, 256), the A-operand layout of the shared-memory tile,
// so one 64 KB bulk copy loads a tile as a tensor-core operand.
struct TrainIO {
    bf16 *H1, *H2, *H3;      // hidden activations (H3 in mode 1 only)
    bf16 *X;                 // the x tiles as multiplied (1 in the padding columns), 4 KB each
    uint32_t *mask1, *mask2; // [tile][slice j][row r]: byte g of the word holds the flags (H_l > 0) of
                             // columns 32 j + 8 g .. + 7 in the order of nz8
    uint32_t *mask3;         // mode 2: the same for H3
    float *dY;               // mode 2: dy per row (0 past M), [tiles * 128]
    const float *target;     // mode 2
    float inv_m;             // 1 / M
    float *gw4, *gb4, *loss; // mode 2: accumulated (atomics)
};
constexpr size_t kTileBytes = 128 * kW * 2, kXTileBytes = 128 * kIn * 2, kMaskTileBytes = 8 * 128 * 4;

// Nonzero flags of the eight BF16 values of q (four pairs, low half first)
// as one byte: bit i for the low half of pair i, bit 4 + i for its high half.
// Per half, bit 15 of (h & 0x7FFF) + 0x7FFF is set iff |h| != 0; for ReLU
// outputs (never negative) that is h > 0.
__device__ __forceinline__ uint32_t nz8(uint4 q)
{
    const uint32_t f0 = (q.x & 0x7FFF7FFFu) + 0x7FFF7FFFu, f1 = (q.y & 0x7FFF7FFFu) + 0x7FFF7FFFu,
                   f2 = (q.z & 0x7FFF7FFFu) + 0x7FFF7FFFu, f3 = (q.w & 0x7FFF7FFFu) + 0x7FFF7FFFu;
    const uint32_t x = ((f0 >> 15) & 0x10001u) | ((f1 >> 14) & 0x20002u) | ((f2 >> 13) & 0x40004u) |
                       ((f3 >> 12) & 0x80008u);
    return (x & 0xFu) | ((x >> 12) & 0xF0u);
}
// 0xFFFF in each half of the pair word w whose BF16 value is nonzero
__device__ __forceinline__ uint32_t nz_halves(uint32_t w)
{
    return ((((w & 0x7FFF7FFFu) + 0x7FFF7FFFu) >> 15) & 0x10001u) * 0xFFFFu;
}
// (a0, a1) * (b0, b1), each lane an IEEE round-to-nearest product, rounded
// to a BF16 pair (low half first)
__device__ __forceinline__ uint32_t bf2_mul_bits(float a0, float a1, float b0, float b1)
{
    uint32_t d;
    asm("{\n\t.reg .b64 a, b, p;\n\t.reg .f32 lo, hi;\n\t"
        "mov.b64 a, {%1, %2};\n\tmov.b64 b, {%3, %4};\n\tmul.rn.f32x2 p, a, b;\n\t"
        "mov.b64 {lo, hi}, p;\n\tcvt.rn.bf16x2.f32 %0, hi, lo;\n\t}"
        : "=r"(d)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
    return d;
}

// kMode 0: inference (y only).  kMode 1: forward for training, also storing
// H1, H2, H3, the x tiles and the ReLU masks of H1 and H2.  kMode 2: the
// forward of a training step: H1, H2, the x tiles and the masks as in mode 1
// (not H3, but its mask), then the head's backward: y, dy = 2 (y - t) / M
// (stored), the loss and the gradients of b4 and w4 (H3^T dy on the tensor
// cores, per tile).  D3 = dy w4 where H3 > 0 is not stored: the kernels that
// use it rebuild it from dy and the mask.  The products and the head's forward arithmetic are those of mode
// 0, so y is bit-identical in all three modes.
template <int kMode>
__global__ void __launch_bounds__(ws::kThreads, 1)
    k_mlp_ws(const bf16 *__restrict__ wh, const float *__restrict__ p, const bf16 *__restrict__ packed,
             const bf16 *__restrict__ x, long long M, const int32_t *__restrict__ count, float *__restrict__ y,
             const TrainIO io)
{
    // rows: M, or the first *count of them when a device count is given
    if (count) {
        const long long c = *count;
        M = c < 0 ? 0 : (c < M ? c : M);
    }
    const long long ntiles = (M + 127) / 128;
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t full[ws::kStages], empty[ws::kStages], xfull[2], xempty[2], accfull[2], accempty[2],
        aready[ws::kChunks], partfull[2], g4ready, g4full, drain;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_fail;
    __shared__ volatile int s_slot[2 + ws::kEpiWarps];
    __shared__ float s_gw4[kMode == 2 ? kW : 1], s_red[2];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    unsigned char *sA = base + ws::oA, *sRing = base + ws::oRing, *sX = base + ws::oX, *sW1 = base + ws::oW1;
    float *sBias = reinterpret_cast<float *>(base + ws::oBias), *sW4 = reinterpret_cast<float *>(base + ws::oW4),
          *sPart = reinterpret_cast<float *>(base + ws::oPart);
    unsigned char *sDY = base + ws::oDY;
    const uint32_t aA = smem_u32(sA), aRing = smem_u32(sRing), aX = smem_u32(sX), aW1 = smem_u32(sW1),
                   aDY = smem_u32(sDY);
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
        tc::mbar_init(&g4ready, ws::kEpiWarps * 32);
        tc::mbar_init(&g4full);
        tc::mbar_init(&drain);
        tc::fence_mbar_init();
        s_fail = 0;
        s_red[0] = s_red[1] = 0.f;
    }
    if (kMode == 2)
        for (int i = tid; i < kW; i += ws::kThreads)
            s_gw4[i] = 0.f;
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
            // mode 2: the w4 gradient of the CTA's tile t, H3^T (dy in three
            // BF16 parts): A = relu(D3 + b3) in the A buffer read MN-major
            // (units M, rows K), B = the dy tile (MN-major, 16 columns), into
            // columns 0..31 of that tile's head accumulator once the epilogue
            // has read it (g4ready)
            auto gw4_products = [&](int t) -> bool {
                if (!tc::mbar_wait(&g4ready, (uint32_t)t & 1u))
                    return false;
                tc::fence_after();
                const uint32_t dcol = tmem + (uint32_t)((3LL * t + 2) & 1) * 256u;
                constexpr uint32_t id = tc::idesc(kIn, true);
#pragma unroll
                for (int s = 0; s < 8; ++s)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        tc::mma_i(dcol + (uint32_t)(h * kIn), tc::sdesc(aA + 8192u * s + 2048u * h, 4096, 128),
                                  tc::sdesc(aDY + 512u * s, 256, 128), id, (uint32_t)(s != 0));
                tc::commit(&g4full);
                return true;
            };
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
                if (kMode == 2 && it > 0 && !gw4_products(it - 1)) {
                    ok = false;
                    break;
                }
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
            if (kMode == 2 && ok && it > 0)
                ok = gw4_products(it - 1);
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
                if constexpr (kMode != 0)
                    *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(io.X) + tile * kXTileBytes +
                                               tc::kmaj(r, h, kIn)) = val;
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
        long long pend = -1;  // tile whose head sums wait to be added (group 0; modes 0 and 1)
        int pend_it = 0;
        float gw4acc = 0.f, gb4acc = 0.f, lossacc = 0.f;  // mode 2 (gw4acc: unit 128 group + r)
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
        auto each_slice = [&](uint32_t tb, auto &&f) { ws::each_slice(tb, group, f); };
        // relu(D + b3) of 8 columns (32 j + 8 g8 ..) as BF16 pairs
        auto relu8 = [&](const uint32_t *u, int j, int g8, uint32_t(&pp)[4]) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float4 b = *reinterpret_cast<const float4 *>(sBias + 2 * kW + 32 * j + 8 * g8 + 4 * h);
                const uint32_t *uu = u + 4 * h;
                pp[2 * h] = bf2_bias_relu_bits(__uint_as_float(uu[0]), __uint_as_float(uu[1]), b.x, b.y);
                pp[2 * h + 1] = bf2_bias_relu_bits(__uint_as_float(uu[2]), __uint_as_float(uu[3]), b.z, b.w);
            }
        };
        // their products with w4 added to the head's four partial sums, each
        // partial sum in column order
        auto dot8 = [&](int j, int g8, const uint32_t(&pp)[4], float(&acc4)[4]) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float4 w = *reinterpret_cast<const float4 *>(sW4 + 32 * j + 8 * g8 + 4 * h);
                const uint32_t p0 = pp[2 * h], p1 = pp[2 * h + 1];
                fma2(acc4[0], acc4[1], __uint_as_float(p0 << 16), __uint_as_float(p0 & 0xffff0000u), w.x, w.y);
                fma2(acc4[2], acc4[3], __uint_as_float(p1 << 16), __uint_as_float(p1 & 0xffff0000u), w.z, w.w);
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
                    uint32_t *mk = nullptr;
                    unsigned char *hst = nullptr;
                    if constexpr (kMode != 0) {
                        mk = (L == 0 ? io.mask1 : io.mask2) + tile * (kMaskTileBytes / 4);
                        hst = reinterpret_cast<unsigned char *>(L == 0 ? io.H1 : io.H2) + tile * kTileBytes;
                    }
                    // slice j (32 columns): bias, ReLU, BF16 into the A operand (modes
                    // 1, 2: and the same 16 bytes into the stored tile, which has the
                    // operand's layout), then its chunk's barrier, then the slice's
                    // mask word; the next slice's load is in flight meanwhile
                    auto slice = [&](const uint32_t(&v)[32], int j, int) {
                        uint4 keep[4];
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
                            const uint32_t off = tc::kmaj(r, 32 * j + 8 * gq, kW);
                            *reinterpret_cast<uint4 *>(sA + off) = pk;
                            if constexpr (kMode != 0)
                                *reinterpret_cast<uint4 *>(hst + off) = pk;
                            keep[gq] = pk;
                        }
                        tc::fence_proxy_async();
                        tc::fence_before();
                        tc::mbar_arrive(&aready[j >> 1]);
                        if constexpr (kMode != 0) {
                            uint32_t bits = 0;
#pragma unroll
                            for (int gq = 0; gq < 4; ++gq)
                                bits |= nz8(keep[gq]) << (8 * gq);
                            mk[j * 128 + r] = bits;
                        }
                    };
                    each_slice(tb, slice);
                    tc::mbar_arrive(&accempty[a]);
                } else if constexpr (kMode == 2) {
                    // head: relu(D + b3) (BF16) into the A buffer, the operand of
                    // the w4 gradient (the third layer's products have read the
                    // buffer), and its dot products with w4
                    float acc4[4] = {0.f, 0.f, 0.f, 0.f};
                    uint32_t *mk3 = io.mask3 + tile * (kMaskTileBytes / 4);
                    auto dot = [&](const uint32_t(&v)[32], int j, int) {
                        uint32_t bits = 0;
#pragma unroll
                        for (int g8 = 0; g8 < 4; ++g8) {
                            uint32_t pp[4];
                            relu8(v + 8 * g8, j, g8, pp);
                            dot8(j, g8, pp, acc4);
                            const uint4 h = make_uint4(pp[0], pp[1], pp[2], pp[3]);
                            *reinterpret_cast<uint4 *>(sA + tc::kmaj(r, 32 * j + 8 * g8, kW)) = h;
                            bits |= nz8(h) << (8 * g8);
                        }
                        mk3[j * 128 + r] = bits;
                    };
                    each_slice(tb, dot);
                    float *part = sPart + (it & 1) * (ws::kGroups * 128);
                    part[group * 128 + r] = (acc4[0] + acc4[1]) + (acc4[2] + acc4[3]);
                    tc::mbar_arrive(&partfull[it & 1]);
                    if (!ws::warp_wait(&partfull[it & 1], (uint32_t)(it >> 1) & 1u, slot, lane)) {
                        ok = false;
                        break;
                    }
                    float sum = 0.f;
#pragma unroll
                    for (int g2 = 0; g2 < ws::kGroups; ++g2)
                        sum += part[g2 * 128 + r];
                    const float yv = sum + b4;
                    const long long m = tile * 128 + r;
                    float dy = 0.f;
                    if (m < M) {
                        const float e = yv - io.target[m];
                        dy = (2.f * e) * io.inv_m;
                        if (group == 0) {
                            y[m] = yv;
                            lossacc += e * e * io.inv_m;
                            gb4acc += dy;
                        }
                    }
                    if (group == 0)
                        io.dY[m] = dy;
                    // row r of the dy tile: dy as three BF16 parts (their sum is
                    // dy to 2^-27 relative: high part, then the high parts of the
                    // remainders) in columns 0..2, zeros elsewhere
                    {
                        uint4 q = make_uint4(0u, 0u, 0u, 0u);
                        if (group == 0) {
                            const __nv_bfloat16 hi = __float2bfloat16_rn(dy);
                            const float r1 = dy - __bfloat162float(hi);
                            const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
                            const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
                            q.x = (uint32_t)__bfloat16_as_ushort(hi) | ((uint32_t)__bfloat16_as_ushort(mid) << 16);
                            q.y = (uint32_t)__bfloat16_as_ushort(lo);
                        }
                        *reinterpret_cast<uint4 *>(sDY + tc::kmaj(r, 8 * group, kIn)) = q;
                    }
                    tc::fence_proxy_async();
                    tc::fence_before();
                    tc::mbar_arrive(&g4ready);
                    // this tile's w4 gradient: unit 128 group + r is lane r of half
                    // `group` (columns 16 group .. 16 group + 2: the three parts)
                    if (!ws::warp_wait(&g4full, (uint32_t)it & 1u, slot, lane)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    {
                        float gv[32];
                        tc::tmem_ld32(tb, gv);
                        gw4acc += group ? (gv[16] + gv[17]) + gv[18] : (gv[0] + gv[1]) + gv[2];
                    }
                    tc::fence_before();
                    tc::mbar_arrive(&accempty[a]);
                } else {
                    // head: relu(D + b3) rounded to BF16 (as stored between layers), . w4,
                    // in four partial sums (mode 1 also stores relu(D + b3) as H3)
                    float acc4[4] = {0.f, 0.f, 0.f, 0.f};
                    unsigned char *h3 = nullptr;
                    if constexpr (kMode == 1)
                        h3 = reinterpret_cast<unsigned char *>(io.H3) + tile * kTileBytes;
                    auto slice = [&](const uint32_t(&v)[32], int j, int) {
#pragma unroll
                        for (int g8 = 0; g8 < 4; ++g8) {
                            uint32_t pp[4];
                            relu8(v + 8 * g8, j, g8, pp);
                            dot8(j, g8, pp, acc4);
                            if constexpr (kMode == 1)
                                *reinterpret_cast<uint4 *>(h3 + tc::kmaj(r, 32 * j + 8 * g8, kW)) =
                                    make_uint4(pp[0], pp[1], pp[2], pp[3]);
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
        if constexpr (kMode == 2) {
            // the CTA's head gradients: one unit per thread, then the groups' rows
            s_gw4[128 * group + r] = gw4acc;
            if (group == 0) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    gb4acc += __shfl_xor_sync(0xffffffffu, gb4acc, o);
                    lossacc += __shfl_xor_sync(0xffffffffu, lossacc, o);
                }
                if (lane == 0) {
                    atomicAdd(&s_red[0], gb4acc);
                    atomicAdd(&s_red[1], lossacc);
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if constexpr (kMode == 2) {
        for (int i = tid; i < kW; i += ws::kThreads)
            atomicAdd(io.gw4 + i, s_gw4[i]);
        if (tid == 0) {
            atomicAdd(io.gb4, s_red[0]);
            if (io.loss)
                atomicAdd(io.loss, s_fail ? __int_as_float(0x7fc00000) : s_red[1]);
        }
    }
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, ws::kCols);
    }
}

// ---------------------------------------------------------------------------
// Input gradients of the hidden layers (after mode 2 of k_mlp_ws): per
// 128-row tile D3 = dy w4 where H3 > 0 (FP32 product rounded to BF16, built
// from the stored dy and mask), D2 = (D3 W3) where H2 > 0 and D1 = (D2 W2)
// where H1 > 0 (FP32 sums rounded to BF16); D2 and D1 are stored packed.
// Persistent and warp-specialised:
//   warp 0 (one thread)  issues the products, B = the packed W3^T and W2^T
//                        chunks (K = the layer's output units);
//   warp 1 (one thread)  producer: the weight chunks through a 3-stage ring;
//   warps 2..9           epilogue: D3 of a tile into its A buffer (two
//                        buffers: tile i uses i % 2; D3 of the next tile is
//                        built while the products D2 W2 of this one run),
//                        then mask and round D2, then D1, into the A buffer;
//                        both go to memory as 64 KB bulk copies (D2 by the
//                        product thread, D1 by one epilogue thread), so the
//                        stores drain while the products run.
// ---------------------------------------------------------------------------
namespace dg {
constexpr int kStages = 3, kEpiWarps = 8, kGroups = kEpiWarps / 4, kSlices = 8 / kGroups,
              kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t oA = 0, oRing = 2 * ws::kBytesA, kEnd = oRing + kStages * ws::kBytesChunk;
constexpr size_t kSmem = 1024 + (size_t)kEnd;
static_assert(kSmem + 2048 <= 227 * 1024, "shared memory");
}  // namespace dg

// BF16 pair of (lo, hi) rounded to nearest even, each half kept where its
// flag is set (flags: bit 0 for lo, bit 16 for hi) and 0 elsewhere
__device__ __forceinline__ uint32_t bf2_masked(uint32_t lo, uint32_t hi, uint32_t flags)
{
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(__uint_as_float(hi)), "f"(__uint_as_float(lo)));
    return d & ((flags & 0x10001u) * 0xFFFFu);
}
// the flags of byte g of a mask word (nz8 order) for pair i at bits i and 16 + i
__device__ __forceinline__ uint32_t pair_flags(uint32_t bits, int g)
{
    const uint32_t mb = (bits >> (8 * g)) & 0xFFu;
    return (mb & 0xFu) | ((mb & 0xF0u) << 12);
}
// D3 of 8 columns (32 j + 8 g ..) of a row: dy w4 (FP32 products rounded to
// BF16) where the mask word's flags are set
__device__ __forceinline__ uint4 d3_8(float dy, uint32_t bits, int g, const float *w)
{
    const uint32_t fl = pair_flags(bits, g);
    const float4 w0 = *reinterpret_cast<const float4 *>(w), w1 = *reinterpret_cast<const float4 *>(w + 4);
    return make_uint4(bf2_mul_bits(dy, dy, w0.x, w0.y) & ((fl & 0x10001u) * 0xFFFFu),
                      bf2_mul_bits(dy, dy, w0.z, w0.w) & (((fl >> 1) & 0x10001u) * 0xFFFFu),
                      bf2_mul_bits(dy, dy, w1.x, w1.y) & (((fl >> 2) & 0x10001u) * 0xFFFFu),
                      bf2_mul_bits(dy, dy, w1.z, w1.w) & (((fl >> 3) & 0x10001u) * 0xFFFFu));
}

__global__ void __launch_bounds__(dg::kThreads, 1)
    k_mlp_dgrad(const bf16 *__restrict__ packedT, const bf16 *__restrict__ w4h, const float *__restrict__ dY,
                const uint32_t *__restrict__ mask3, const uint32_t *__restrict__ mask2,
                const uint32_t *__restrict__ mask1, bf16 *__restrict__ D2, bf16 *__restrict__ D1, long long ntiles,
                float *__restrict__ fail_sink)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t full[dg::kStages], empty[dg::kStages], accfull[2], accempty[2], d3ready[ws::kChunks],
        aready[ws::kChunks], esync, drain;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_fail;
    __shared__ volatile int s_slot[2 + dg::kEpiWarps];
    __shared__ __align__(16) float sW4[kW];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    unsigned char *sA = base + dg::oA, *sRing = base + dg::oRing;
    const uint32_t aA = smem_u32(sA), aRing = smem_u32(sRing);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0)
        tc::tmem_alloc(&s_tmem, ws::kCols);
    if (tid == 0) {
        for (int i = 0; i < dg::kStages; ++i) {
            tc::mbar_init(&full[i]);
            tc::mbar_init(&empty[i]);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&accfull[i]);
            tc::mbar_init(&accempty[i], dg::kEpiWarps * 32);
        }
        for (int j = 0; j < ws::kChunks; ++j) {
            tc::mbar_init(&d3ready[j], 2 * 4 * 32);  // two slices, each written by the four warps of its group
            tc::mbar_init(&aready[j], 2 * 4 * 32);
        }
        tc::mbar_init(&esync, dg::kEpiWarps * 32);
        tc::mbar_init(&drain);
        tc::fence_mbar_init();
        s_fail = 0;
    }
    for (int i = tid; i < kW; i += dg::kThreads)
        sW4[i] = __bfloat162float(w4h[i]);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        // ---- products: tile it uses A buffer it % 2; q = 2 it + layer ------
        if (lane == 0) {
            long long g = 0;
            bool ok = true;
            int it = 0;
            for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
                const int b = it & 1;
                for (int L = 0; L < 2 && ok; ++L) {
                    const long long q = 2LL * it + L;
                    const uint32_t dcol = tmem + (uint32_t)(q & 1) * 256u;
                    if (q >= 2 && !tc::mbar_wait(&accempty[q & 1], (uint32_t)((q - 2) >> 1) & 1u)) {
                        ok = false;
                        break;
                    }
                    for (int c = 0; c < ws::kChunks; ++c, ++g) {
                        const int st = (int)(g % dg::kStages);
                        if (!tc::mbar_wait(&full[st], (uint32_t)(g / dg::kStages) & 1u) ||
                            !tc::mbar_wait(L == 0 ? &d3ready[c] : &aready[c], (uint32_t)it & 1u)) {
                            ok = false;
                            break;
                        }
                        if (L == 1 && c == ws::kChunks - 1)  // D2 complete in the A buffer: to memory
                            tc::bulk_store(reinterpret_cast<unsigned char *>(D2) + tile * kTileBytes,
                                           sA + b * ws::kBytesA, ws::kBytesA);
                        tc::fence_after();
#pragma unroll
                        for (int kk = 0; kk < tc::kKC / 16; ++kk) {
                            const int k0 = tc::kKC * c + 16 * kk;
                            tc::mma(dcol, tc::sdesc(aA + (uint32_t)b * ws::kBytesA + (uint32_t)(k0 / 8) * 128u, 128, kW * 16),
                                    tc::sdesc(aRing + (uint32_t)(st * ws::kBytesChunk + kk * 256), 128, tc::kKC * 16),
                                    (uint32_t)(c | kk));
                        }
                        tc::commit(&empty[st]);
                    }
                    // the epilogue writes D1 into the A buffer once this
                    // accumulator is full: the copy of D2 has read it by then
                    if (L == 1)
                        tc::bulk_wait_read();
                    if (ok)
                        tc::commit(&accfull[q & 1]);
                }
                if (s_fail)
                    ok = false;
            }
            if (!ok)
                s_fail = 1;
            tc::bulk_wait_all();
            tc::commit(&drain);
            (void)tc::mbar_wait(&drain, 0);
        }
    } else if (warp == 1) {
        // ---- producer ------------------------------------------------------
        if (lane == 0) {
            long long g = 0;
            bool ok = true;
            for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                for (int c = 0; c < 2 * ws::kChunks; ++c, ++g) {
                    const int st = (int)(g % dg::kStages);
                    if (s_fail ||
                        (g >= dg::kStages && !tc::mbar_wait(&empty[st], (uint32_t)(g / dg::kStages - 1) & 1u))) {
                        s_fail = 1;
                        ok = false;
                        break;
                    }
                    tc::bulk_load(sRing + st * ws::kBytesChunk, packedT + (long long)c * (kW * tc::kKC),
                                  ws::kBytesChunk, &full[st]);
                }
            }
            // copies still in flight are among the last kStages issued
            for (long long c = g > dg::kStages ? g - dg::kStages : 0; c < g; ++c)
                (void)tc::mbar_wait(&full[c % dg::kStages], (uint32_t)(c / dg::kStages) & 1u);
        }
    } else {
        // ---- epilogue ------------------------------------------------------
        const int quarter = warp & 3, group = (warp - 2) >> 2;
        const int r = quarter * 32 + lane;
        volatile int *slot = s_slot + warp;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        // the epilogue warps alone meet (a bounded wait; its phases alternate)
        bool ok = true;
        int nsync = 0;
        auto epi_sync = [&] {
            tc::mbar_arrive(&esync);
            if (!ws::warp_wait(&esync, (uint32_t)(nsync++ & 1), slot, lane))
                ok = false;
        };
        // dy and the H3 mask words of tile t for this thread's row and slices
        float ndy = 0.f;
        uint32_t nm3[dg::kSlices];
        auto fetch_d3 = [&](long long t) {
            ndy = dY[t * 128 + r];
#pragma unroll
            for (int k = 0; k < dg::kSlices; ++k)
                nm3[k] = mask3[t * (kMaskTileBytes / 4) + (group + k * dg::kGroups) * 128 + r];
        };
        // D3 of the fetched tile into A buffer b, each slice's chunk barrier once
        // written; the copy of D1 out of that buffer (two tiles before) has read
        // it first
        auto build_d3 = [&](int b) {
            if (warp == 2 && lane == 0)
                tc::bulk_wait_read();
            epi_sync();
            unsigned char *sa = sA + b * ws::kBytesA;
#pragma unroll
            for (int k = 0; k < dg::kSlices; ++k) {
                const int j = group + k * dg::kGroups;
#pragma unroll
                for (int g = 0; g < 4; ++g)
                    *reinterpret_cast<uint4 *>(sa + tc::kmaj(r, 32 * j + 8 * g, kW)) =
                        d3_8(ndy, nm3[k], g, sW4 + 32 * j + 8 * g);
                tc::fence_proxy_async();
                tc::fence_before();
                tc::mbar_arrive(&d3ready[j >> 1]);
            }
        };
        int it = 0;
        long long tile = blockIdx.x;
        if (tile < ntiles) {
            fetch_d3(tile);
            build_d3(0);
        }
        for (; tile < ntiles; tile += gridDim.x, ++it) {
            const int b = it & 1;
            const bool more = tile + gridDim.x < ntiles;
            uint32_t m2[dg::kSlices], m1[dg::kSlices];
#pragma unroll
            for (int k = 0; k < dg::kSlices; ++k) {
                const long long o = tile * (kMaskTileBytes / 4) + (group + k * dg::kGroups) * 128 + r;
                m2[k] = mask2[o];
                m1[k] = mask1[o];
            }
            if (more)
                fetch_d3(tile + gridDim.x);
            for (int L = 0; L < 2 && ok; ++L) {
                const long long q = 2LL * it + L;
                const int a = (int)(q & 1);
                if (!ws::warp_wait(&accfull[a], (uint32_t)(q >> 1) & 1u, slot, lane)) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                const uint32_t tb = tmem + (uint32_t)a * 256u + lane_off;
                unsigned char *sa = sA + b * ws::kBytesA;
                // D2 (then D1) into the A buffer: D2 is the next products' operand
                // (each chunk's barrier releases them) and the product thread copies
                // it to memory; D1 goes to memory from the buffer below
                auto slice = [&](const uint32_t(&v)[32], int j, int k) {
                    const uint32_t bits = L == 0 ? m2[k] : m1[k];
#pragma unroll
                    for (int gq = 0; gq < 4; ++gq) {
                        const uint32_t *u = v + 8 * gq;
                        const uint32_t fl = pair_flags(bits, gq);
                        uint4 pk;
                        pk.x = bf2_masked(u[0], u[1], fl);
                        pk.y = bf2_masked(u[2], u[3], fl >> 1);
                        pk.z = bf2_masked(u[4], u[5], fl >> 2);
                        pk.w = bf2_masked(u[6], u[7], fl >> 3);
                        *reinterpret_cast<uint4 *>(sa + tc::kmaj(r, 32 * j + 8 * gq, kW)) = pk;
                    }
                    tc::fence_proxy_async();
                    if (L == 0) {
                        tc::fence_before();
                        tc::mbar_arrive(&aready[j >> 1]);
                    }
                };
                ws::each_slice<dg::kGroups>(tb, group, slice);
                tc::fence_before();
                tc::mbar_arrive(&accempty[a]);
                if (L == 1) {
                    // D1 complete in the buffer (all epilogue warps): one thread
                    // copies it to memory; the buffer is next written two tiles on
                    epi_sync();
                    if (warp == 2 && lane == 0)
                        tc::bulk_store(reinterpret_cast<unsigned char *>(D1) + tile * kTileBytes, sa, ws::kBytesA);
                }
                // the next tile's D3 goes into the other buffer while this tile's
                // second products run (its last reader, the products of the tile
                // before, finished before that tile's D1 was read)
                if (L == 0 && more)
                    build_d3(b ^ 1);
            }
            if (!ok || ws::warp_uniform(s_fail, slot, lane))
                break;
        }
        if (!ok)
            s_fail = 1;
        if (warp == 2 && lane == 0)
            tc::bulk_wait_all();
    }
    tc::fence_before();
    __syncthreads();
    if (tid == 0 && s_fail)
        atomicAdd(fail_sink, __int_as_float(0x7fc00000));
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, ws::kCols);
    }
}

// ---------------------------------------------------------------------------
// Weight and bias gradients (after k_mlp_dgrad): grad W_l += D_l^T H_{l-1}
// and grad b_l += the column sums of D_l, H_0 the x tiles as multiplied.  One
// CTA per job: a layer (3, 2 or 1) and a contiguous range of tiles.  Both
// operands are the packed tiles read as MN-major (transposed) operands: the
// rows of the batch are K, D_l's columns (output units) M, H's columns N.
// Per 32-row piece, two k16 steps of two M = 128 products (output units
// 0..127 and 128..255) into two FP32 accumulators of 256 columns (16 for the
// first layer) in tensor memory.  Roles:
//   warp 0 (one thread)  the products;
//   warp 1 (one thread)  producer: the D and H (or x) pieces through a
//                        6-stage ring, two bulk copies on one barrier (the H2
//                        piece alone for the third layer);
//   warps 2..9           third layer: build each D3 piece in the ring from
//                        dy, the mask of H3 and w4 (warp w: columns 32 w ..);
//                        all layers: while the products run, the column sums
//                        of each D piece from shared memory (FP32); at the
//                        end the accumulators (tcgen05.ld) into the gradient
//                        with vector atomics.
// The padding columns 13..15 of the first layer's gradient are not written.
// ---------------------------------------------------------------------------
namespace wg {
constexpr int kStages = 6, kSumWarps = 8, kThreads = 32 * (2 + kSumWarps);
constexpr uint32_t kPiece = 32 * kW * 2;   // 32 rows of a packed tile (16 KB)
constexpr uint32_t kXPiece = 32 * kIn * 2; // 32 rows of a packed x tile (1 KB)
constexpr uint32_t kDy = 2 * kPiece, kMask = kDy + 32 * 4;  // third layer: dy and mask words of a piece
constexpr uint32_t kStage = kMask + 8 * 32 * 4;
constexpr size_t kSmem = 1024 + (size_t)kStages * kStage;
static_assert(kSmem + 1024 <= 227 * 1024, "shared memory");
}  // namespace wg

struct WgradArgs {
    const float *dY;          // dy per row
    const uint32_t *mask3;    // ReLU mask of H3
    const bf16 *w4h;          // BF16 head weights
    const bf16 *D2, *D1, *H2, *H1, *X;
    float *g;         // gradient vector (parameter order)
    long long ntiles;
    int jobs3, jobs2, jobs1;  // jobs per layer, each at most ntiles
};

__global__ void __launch_bounds__(wg::kThreads, 1) k_mlp_wgrad(const WgradArgs A)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t full[wg::kStages], empty[wg::kStages], dfull[wg::kStages], accfull, drain;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_fail;
    __shared__ volatile int s_slot[2 + wg::kSumWarps];
    __shared__ __align__(16) float sW4[kW];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t aS = smem_u32(base);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    int layer, j, J;
    if ((int)blockIdx.x < A.jobs3) {
        layer = 3, j = blockIdx.x, J = A.jobs3;
    } else if ((int)blockIdx.x < A.jobs3 + A.jobs2) {
        layer = 2, j = blockIdx.x - A.jobs3, J = A.jobs2;
    } else {
        layer = 1, j = blockIdx.x - A.jobs3 - A.jobs2, J = A.jobs1;
    }
    const long long t0 = A.ntiles * j / J, t1 = A.ntiles * (j + 1) / J;
    const long long np = 4 * (t1 - t0);  // 32-row pieces
    const bool wide = layer != 1, build = layer == 3;  // build: D3 made in shared memory
    const unsigned char *Dp = reinterpret_cast<const unsigned char *>(layer == 2 ? A.D2 : A.D1);
    const unsigned char *Hp = reinterpret_cast<const unsigned char *>(layer == 3 ? A.H2 : layer == 2 ? A.H1 : A.X);
    const uint32_t hbytes = wide ? wg::kPiece : wg::kXPiece;
    const size_t htile = wide ? kTileBytes : kXTileBytes;
    float *gW = A.g + (layer == 3 ? oW3 : layer == 2 ? oW2 : oW1);
    float *gb = A.g + (layer == 3 ? oB3 : layer == 2 ? oB2 : oB1);

    if (warp == 0)
        tc::tmem_alloc(&s_tmem, ws::kCols);
    if (tid == 0) {
        for (int i = 0; i < wg::kStages; ++i) {
            // full: the copies, or for the third layer the eight builders (who
            // wait for the copies on dfull first)
            tc::mbar_init(&full[i], build ? wg::kSumWarps : 1);
            tc::mbar_init(&empty[i], 1 + wg::kSumWarps);  // the products' commit and the summing warps
            tc::mbar_init(&dfull[i]);
        }
        tc::mbar_init(&accfull);
        tc::mbar_init(&drain);
        tc::fence_mbar_init();
        s_fail = 0;
    }
    for (int i = tid; i < kW; i += wg::kThreads)
        sW4[i] = __bfloat162float(A.w4h[i]);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        // ---- products ------------------------------------------------------
        if (lane == 0 && np > 0) {
            const uint32_t ncol = wide ? kW : kIn, id = tc::idesc((int)ncol, true);
            for (long long p = 0; p < np; ++p) {
                const int st = (int)(p % wg::kStages);
                if (!tc::mbar_wait(&full[st], (uint32_t)(p / wg::kStages) & 1u)) {
                    s_fail = 1;
                    break;
                }
                tc::fence_after();
                const uint32_t sa = aS + (uint32_t)st * wg::kStage, sb = sa + wg::kPiece;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    // K = rows: 8-row groups 4096 bytes apart in D and H, 256 in x;
                    // M (N) = units: 8-unit groups 128 bytes apart
                    const uint64_t db = wide ? tc::sdesc(sb + 8192u * s, 4096, 128) : tc::sdesc(sb + 512u * s, 256, 128);
#pragma unroll
                    for (int a = 0; a < 2; ++a)
                        tc::mma_i(tmem + (uint32_t)a * ncol, tc::sdesc(sa + 8192u * s + 2048u * a, 4096, 128), db, id,
                                  (uint32_t)((p | s) != 0));
                }
                tc::commit(&empty[st]);
            }
            tc::commit(&accfull);
            tc::commit(&drain);
            (void)tc::mbar_wait(&drain, 0);
        }
    } else if (warp == 1) {
        // ---- producer ------------------------------------------------------
        if (lane == 0) {
            long long p = 0;
            for (; p < np; ++p) {
                const int st = (int)(p % wg::kStages);
                if (s_fail ||
                    (p >= wg::kStages && !tc::mbar_wait(&empty[st], (uint32_t)(p / wg::kStages - 1) & 1u))) {
                    s_fail = 1;
                    break;
                }
                const long long tile = t0 + p / 4;
                const int pc = (int)(p % 4);
                unsigned char *dst = base + (size_t)st * wg::kStage;
                if (build) {
                    // the H2 piece, the piece's dy and its mask words (eight runs of 32)
                    uint64_t *bar = &dfull[st];
                    tc::expect_tx(bar, hbytes + 32 * 4 + 8 * 32 * 4);
                    tc::bulk_copy(dst + wg::kPiece, Hp + tile * htile + (size_t)pc * hbytes, hbytes, bar);
                    tc::bulk_copy(dst + wg::kDy, A.dY + tile * 128 + pc * 32, 32 * 4, bar);
                    for (int j = 0; j < 8; ++j)
                        tc::bulk_copy(dst + wg::kMask + j * 128,
                                      A.mask3 + tile * (kMaskTileBytes / 4) + j * 128 + pc * 32, 32 * 4, bar);
                } else {
                    tc::expect_tx(&full[st], wg::kPiece + hbytes);
                    tc::bulk_copy(dst, Dp + tile * kTileBytes + (size_t)pc * wg::kPiece, wg::kPiece, &full[st]);
                    tc::bulk_copy(dst + wg::kPiece, Hp + tile * htile + (size_t)pc * hbytes, hbytes, &full[st]);
                }
            }
            for (long long c = p > wg::kStages ? p - wg::kStages : 0; c < p; ++c)
                (void)tc::mbar_wait(build ? &dfull[c % wg::kStages] : &full[c % wg::kStages],
                                    (uint32_t)(c / wg::kStages) & 1u);
        }
    } else {
        // ---- column sums, then the accumulators ----------------------------
        const int w = warp - 2, ri = lane & 7, kg = (lane >> 3) + 4 * w;  // row in group, column group
        volatile int *slot = s_slot + warp;
        float cs[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            cs[i] = 0.f;
        bool ok = true;
        for (long long p = 0; p < np; ++p) {
            const int st = (int)(p % wg::kStages);
            unsigned char *sa = base + (size_t)st * wg::kStage;
            if (build) {
                // D3 rows 32 pc .. of the tile, columns 32 w .. (this warp's
                // slice), from the piece's dy and mask words in the stage (the
                // producer copies them once the slot's products and readers
                // are done)
                if (!ws::warp_wait(&dfull[st], (uint32_t)(p / wg::kStages) & 1u, slot, lane)) {
                    ok = false;
                    break;
                }
                const float dy = reinterpret_cast<const float *>(sa + wg::kDy)[lane];
                const uint32_t bits = reinterpret_cast<const uint32_t *>(sa + wg::kMask)[w * 32 + lane];
#pragma unroll
                for (int g = 0; g < 4; ++g)
                    *reinterpret_cast<uint4 *>(sa + tc::kmaj(lane, 32 * w + 8 * g, kW)) =
                        d3_8(dy, bits, g, sW4 + 32 * w + 8 * g);
                __syncwarp();
            } else if (!ws::warp_wait(&full[st], (uint32_t)(p / wg::kStages) & 1u, slot, lane)) {
                ok = false;
                break;
            }
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const uint4 q = *reinterpret_cast<const uint4 *>(sa + g * 4096 + kg * 128 + ri * 16);
                const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    cs[2 * i] += __uint_as_float(u[i] << 16);
                    cs[2 * i + 1] += __uint_as_float(u[i] & 0xffff0000u);
                }
            }
            if (build) {
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0)
                    tc::mbar_arrive(&full[st]);
            }
            __syncwarp();
            if (lane == 0)
                tc::mbar_arrive(&empty[st]);
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1)
#pragma unroll
            for (int i = 0; i < 8; ++i)
                cs[i] += __shfl_xor_sync(0xffffffffu, cs[i], o);
        if (ok && ri == 0)
#pragma unroll
            for (int i = 0; i < 8; ++i)
                atomicAdd(gb + kg * 8 + i, cs[i]);
        if (ok && np > 0) {
            ok = ws::warp_wait(&accfull, 0, slot, lane) && !ws::warp_uniform(s_fail, slot, lane);
            if (ok) {
                tc::fence_after();
                const int quarter = warp & 3, half = w >> 2;
                const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
                const int n = 128 * half + 32 * quarter + lane;  // output unit of this lane
                if (wide) {
                    for (int c = 0; c < kW / 32; ++c) {
                        float v[32];
                        tc::tmem_ld32(tl + (uint32_t)(half * kW + 32 * c), v);
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            atomicAdd(reinterpret_cast<float4 *>(gW + (long long)n * kW + 32 * c + 4 * i),
                                      make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]));
                    }
                } else {
                    float v[32];  // columns 0..15: output units 0..127, 16..31: 128..255
                    tc::tmem_ld32(tl, v);
#pragma unroll
                    for (int k = 0; k < PCDF_MLP_IN; ++k)
                        atomicAdd(gW + n * kIn + k, half ? v[16 + k] : v[k]);
                }
            }
        }
        if (!ok)
            s_fail = 1;
    }
    tc::fence_before();
    __syncthreads();
    if (tid == 0 && s_fail)
        atomicAdd(A.g + oB4, __int_as_float(0x7fc00000));
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, ws::kCols);
    }
}

// ---------------------------------------------------------------------------
// Adam, initialisation
// ---------------------------------------------------------------------------
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
    bf16 *h, *pk;  // BF16 weights; W2, W3, W3^T, W2^T packed for the tensor-core kernels
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

// refreshes the packed copies of the hidden weights after the BF16 weights change
__global__ void k_pack_hidden(const bf16 *__restrict__ wh, bf16 *__restrict__ packed);
cudaError_t launch_pack(const State &S, cudaStream_t st)
{
    k_pack_hidden<<<(4 * kW * (kW / 8) + 255) / 256, 256, 0, st>>>(S.h, S.pk);
    return cudaGetLastError();
}

// Workspace sections, in this order, for T = ceil(M / 128) tiles: H1, H2, H3,
// D2, D1 (T x 64 KB each, tiles packed as in TrainIO), the x tiles as
// multiplied (T x 4 KB), the ReLU masks of H1, H2 and H3 (T x 4 KB each) and
// dy (T x 512 bytes); see pcdf_mlp_backward.
struct Acts {
    bf16 *H1, *H2, *H3, *D2, *D1, *X;
    uint32_t *mask1, *mask2, *mask3;
    float *dY;
};

size_t ws_bytes(long long M)
{
    const size_t T = (size_t)((M + 127) / 128);
    return T * (5 * kTileBytes + kXTileBytes + 3 * kMaskTileBytes + 128 * sizeof(float));
}

Acts carve(void *ws, long long M)
{
    char *b = (char *)ws;
    const size_t T = (size_t)((M + 127) / 128), a = T * kTileBytes, m = T * kMaskTileBytes;
    Acts r;
    r.H1 = (bf16 *)b;
    r.H2 = (bf16 *)(b + a);
    r.H3 = (bf16 *)(b + 2 * a);
    r.D2 = (bf16 *)(b + 3 * a);
    r.D1 = (bf16 *)(b + 4 * a);
    r.X = (bf16 *)(b + 5 * a);
    char *mk = b + 5 * a + T * kXTileBytes;
    r.mask1 = (uint32_t *)mk;
    r.mask2 = (uint32_t *)(mk + m);
    r.mask3 = (uint32_t *)(mk + 2 * m);
    r.dY = (float *)(mk + 3 * m);
    return r;
}

cudaError_t sm_count(int *nsm)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, dev);
    return e;
}

// the persistent forward kernel: one CTA per SM (or per tile, if fewer)
template <int kMode>
cudaError_t launch_ws(const State &S, const bf16 *x, long long M, const int32_t *count, float *y, const TrainIO &io,
                      cudaStream_t st)
{
    int nsm = 0;
    cudaError_t e = sm_count(&nsm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_ws<kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws::kSmem);
    if (e != cudaSuccess)
        return e;
    const long long ntiles = (M + 127) / 128;
    k_mlp_ws<kMode><<<(unsigned)(ntiles < nsm ? ntiles : nsm), ws::kThreads, ws::kSmem, st>>>(S.h, S.p, S.pk, x, M,
                                                                                             count, y, io);
    return cudaGetLastError();
}

// the input and weight gradients after mode 2 of the forward kernel
cudaError_t launch_backward(const State &S, const Acts &A, long long M, cudaStream_t st)
{
    int nsm = 0;
    cudaError_t e = sm_count(&nsm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_dgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dg::kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wg::kSmem);
    if (e != cudaSuccess)
        return e;
    const long long T = (M + 127) / 128;
    k_mlp_dgrad<<<(unsigned)(T < nsm ? T : nsm), dg::kThreads, dg::kSmem, st>>>(
        S.pk + 2 * kW * kW, S.h + hW4, A.dY, A.mask3, A.mask2, A.mask1, A.D2, A.D1, T, S.g + oB4);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    // jobs in proportion to the time a tile takes, measured: the second layer
    // streams D2 and H1 (128 KB), the third H2 with dy and the mask (68 KB)
    // and builds D3 on chip, which costs about as much; the first streams D1
    // and x (68 KB)
    WgradArgs W;
    W.dY = A.dY;
    W.mask3 = A.mask3;
    W.w4h = S.h + hW4;
    W.D2 = A.D2;
    W.D1 = A.D1;
    W.H2 = A.H2;
    W.H1 = A.H1;
    W.X = A.X;
    W.g = S.g;
    W.ntiles = T;
    const int j3 = std::max(1, nsm * 128 / 324), j2 = j3, j1 = std::max(1, nsm - j3 - j2);
    W.jobs3 = (int)std::min<long long>(j3, T);
    W.jobs2 = (int)std::min<long long>(j2, T);
    W.jobs1 = (int)std::min<long long>(j1, T);
    k_mlp_wgrad<<<(unsigned)(W.jobs3 + W.jobs2 + W.jobs1), wg::kThreads, wg::kSmem, st>>>(W);
    return cudaGetLastError();
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
    TrainIO io;
    std::memset(&io, 0, sizeof(io));
    const cudaError_t e = launch_ws<0>(S, (const bf16 *)x, M, count, y, io, (cudaStream_t)stream);
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
    const Acts A = carve(workspace, M);
    TrainIO io;
    std::memset(&io, 0, sizeof(io));
    io.H1 = A.H1;
    io.H2 = A.H2;
    io.H3 = A.H3;
    io.X = A.X;
    io.mask1 = A.mask1;
    io.mask2 = A.mask2;
    const cudaError_t e = launch_ws<1>(S, (const bf16 *)x, M, nullptr, y, io, (cudaStream_t)stream);
    return e == cudaSuccess ? PCDF_OK : cuda_fail(e, "mlp forward");
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
    const Acts A = carve(workspace, M);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(S.g, 0, 4 * kPpad, st);
    if (e == cudaSuccess && loss)
        e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess)
        return cuda_fail(e, "mlp backward reset");
    TrainIO io;
    std::memset(&io, 0, sizeof(io));
    io.H1 = A.H1;
    io.H2 = A.H2;
    io.X = A.X;
    io.mask1 = A.mask1;
    io.mask2 = A.mask2;
    io.mask3 = A.mask3;
    io.dY = A.dY;
    io.target = target;
    io.inv_m = 1.f / (float)M;
    io.gw4 = S.g + oW4;
    io.gb4 = S.g + oB4;
    io.loss = loss;
    e = launch_ws<2>(S, (const bf16 *)x, M, nullptr, y, io, st);
    if (e == cudaSuccess)
        e = launch_backward(S, A, M, st);
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
