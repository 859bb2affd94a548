// Many environments of uneven size, horizon and human count in one
// persistent launch (sm_103a).
//
// Every environment needs the static field (row words, the fused x+y pass and
// the z pass of edt_full.cuh, the last also recording each column's largest
// value) and its T composite fields
// (capsule x+y pass over the slab, fused z pass).  The host cuts all of that
// into work items (environment, stage, tile).  The first persistent launch
// takes the row-pass, capsule, y and z items from a global queue in that
// order; the second takes the composite items (column block, time steps),
// which run the single-environment kernel's shortcuts: columns whose static
// maximum no human can undercut are copies, blocks of such columns are copied
// with 16-byte accesses, and the envelope is evaluated only in the z window
// around the slab.  Two launches let each have its own register and shared
// memory budget.  An item whose inputs come from an earlier stage of the same
// environment waits (one thread, bounded spin, acquire loads) until the
// completion counter of that stage reaches the stage's item count; finished
// items publish with a release increment.  Because an item only ever waits for
// items that were taken from the queue before it, by CTAs that are already
// running, the queue always drains, whatever the number of resident CTAs.
// A wait that exceeds its bound sets an error word, counts the item as done
// and skips it; the host reads the word with pcdf_batch_error.
//
// The launch needs no host synchronisation and no allocation, so it can be
// captured in a CUDA graph together with the counter reset.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "composite.cuh"
#include "edt_full.cuh"
#include "host.h"

using namespace pcdf::host;

namespace pcdf {
namespace {

constexpr int kThreads = 128;
constexpr int kBands = kThreads / lean::kCols;  // envelope threads per column
constexpr long long kSpinLimit = 1LL << 22;  // x 256 ns sleep: about one second

enum ItemType : int { kRow = 0, kY = 1, kZ = 2, kDyn = 3, kComp = 4 };

struct BatchItem {
    int type, env, a, b;
};

struct BatchEnv {
    int nx, ny, nz, T, H, zlo, S, cap, W;
    float vox;
    int need[4];  // items of the row, y, z and capsule stages
    int vec;      // 16-byte copies of all-static column blocks allowed
    const uint8_t *occ;
    int32_t *comp_sq;
    uint32_t *bits;   // row words, [nz][ny][W]
    uint2 *carry;     // their carries, [nz][ny][W]
    int32_t *mid;
    int32_t *static_sq;
    int32_t *colmax;  // [ny][nx] largest static value of each column
    int32_t *dyn;
    const uint8_t *rep;   // [T][S] slab slice map (slices of equal capsule cross-sections); NULL: identity
    const CapInfo *caps;  // [T][H]
};

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void add_release(int *p, int v)
{
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *p >= target.  Gives up after about a second, or at once when an
// earlier wait has already failed, so a broken dependency cannot keep the
// kernel alive for long.
__device__ bool wait_ge(const int *p, int target, int *err)
{
    for (long long i = 0; i < kSpinLimit; ++i) {
        if (ld_acquire(p) >= target)
            return true;
        if ((i & 255) == 0 && ld_acquire(err) != 0)
            return false;
        __nanosleep(256);
    }
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ void run_rows(const BatchEnv &E, int r0, int r1)
{
    const int lane = threadIdx.x & 31;
    for (int r = r0 + (threadIdx.x >> 5); r < r1; r += kThreads / 32)
        full::row_bits_row<0>(E.occ, nullptr, 0, E.nx, E.ny, r, (long long)E.ny * E.nz, E.W, E.bits, E.carry, lane);
}

// 5 CTAs per SM: the envelope stages' shared memory (up to 42 KB at 320-voxel
// axes) allows no more, and the register budget that follows keeps spills
// to a few words
__global__ void __launch_bounds__(kThreads, 5)
    k_batched(const BatchEnv *__restrict__ envs, const BatchItem *__restrict__ items, int n_items, int *state,
              int row_rows, int dyn_slices, int comp_t)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int s_item, s_ok;
    int *head = state, *err = state + 1, *ctr = state + 2;  // ctr[4 * env + stage]
    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items)
            break;
        const BatchItem I = items[it];
        const BatchEnv &E = envs[I.env];
        int *ce = ctr + 4 * I.env;
        if (threadIdx.x == 0) {
            bool ok = true;
            if (I.type == kY)
                ok = wait_ge(ce + kRow, E.need[kRow], err);
            else if (I.type == kZ)
                ok = wait_ge(ce + kY, E.need[kY], err);
            s_ok = ok;
        }
        __syncthreads();
        if (s_ok) {
            switch (I.type) {
            case kRow:
                run_rows(E, I.a, min(I.a + row_rows, E.ny * E.nz));
                break;
            case kY:  // slice I.a, row word I.b
                full::edt_xy_block<kBands, true>(E.bits, E.carry, E.nx, E.ny, E.nz, E.W, I.b, I.a, E.mid, smem);
                break;
            case kZ:
                full::edt_z_block<kBands, false, true>(E.mid, E.static_sq, nullptr, 0.f, E.nz,
                                                       (long long)E.nx * E.ny, (long long)I.a, smem, E.colmax);
                break;
            case kDyn: {  // time I.a, slices from I.b / 16, column block I.b % 16
                const int s0 = I.b >> 4, x0 = (I.b & 15) * kThreads;
                for (int s = s0; s < min(s0 + dyn_slices, E.S); ++s) {
                    if (E.rep && E.rep[I.a * E.S + s] != s)
                        continue;  // read from the earlier slice of equal cross-sections
                    comp::dyn_xy_slice(E.caps + (long long)I.a * E.H, E.H, E.nx, E.ny, E.zlo, E.S, I.a, s, E.cap,
                                       E.dyn, reinterpret_cast<int32_t *>(smem), x0, min(x0 + kThreads, E.nx));
                    __syncthreads();
                }
                break;
            }
            default:
                break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            add_release(ce + I.type, 1);
        }
    }
}

// The composite items, after every static and capsule item has finished (the
// previous launch on the stream): item (env, t, column block) computes time
// steps t .. t + comp_t - 1 of 128 consecutive columns.  Nothing to wait for;
// if a dependency wait of the first launch expired, the items are skipped.
__global__ void __launch_bounds__(kThreads)
    k_batched_comp(const BatchEnv *__restrict__ envs, const BatchItem *__restrict__ items, int n_items,
                   const int *__restrict__ err, int *head, int comp_t)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int s_item;
    if (*err != 0)
        return;  // uniform: every thread reads the same word
    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items)
            break;
        const BatchItem I = items[it];
        const BatchEnv &E = envs[I.env];
        // the items of a column block (one per group of comp_t steps) split
        // the L2 prefetch of its static columns, before their first step
        const int ngroups = (E.T + comp_t - 1) / comp_t;
        for (int t = I.a; t < min(I.a + comp_t, E.T); ++t) {
            comp::composite_block_short<true, false, false>(E.static_sq, nullptr, E.colmax, E.dyn,
                                                            E.rep ? E.rep + t * E.S : nullptr, E.nx, E.ny, E.nz,
                                                            E.zlo, E.S, t, (long long)I.b, E.comp_sq, nullptr,
                                                            E.vox, E.vec != 0, smem, I.a / comp_t,
                                                            t == I.a && E.vec ? ngroups : 0);
            __syncthreads();
        }
    }
}

// shared memory words of the first launch's stages, and of a composite item
size_t smem_words_env(const CompositePlan &p, const pcdf_grid &g, int H)
{
    auto col = [](int n) { return (size_t)lean::kCols * (n + (n + 31) / 32); };
    size_t w = std::max(col(g.ny), col(g.nz));
    if (p.S > 0)
        w = std::max(w, (size_t)g.ny * (H + 1) + (size_t)p.cap * kThreads);
    return w;
}
size_t smem_words_comp(const CompositePlan &p) { return (size_t)kThreads * (p.S + 2 + (p.S + 31) / 32); }

}  // namespace
}  // namespace pcdf

struct pcdf_batch {
    pcdf_batch_tiles tiles;
    int n_env = 0;
    std::vector<pcdf_env> user;
    std::vector<pcdf::host::CompositePlan> plans;
    std::vector<pcdf::BatchEnv> desc;   // device pointers filled at upload
    std::vector<size_t> off_bits, off_carry, off_mid, off_static, off_colmax, off_dyn, off_caps, off_rep;
    std::vector<pcdf::BatchItem> items;  // the first launch's items, then the composite items
    int n_first = 0;                     // items of the first launch
    size_t off_desc = 0, off_items = 0, off_state = 0, bytes = 0;
    size_t smem = 0, smem_comp = 0;
    int blocks = 0, blocks_comp = 0;
};

namespace {

void default_tiles(pcdf_batch_tiles &t)
{
    if (t.row_rows <= 0)
        t.row_rows = 32;
    if (t.dyn_slices <= 0)
        t.dyn_slices = 1;
    if (t.comp_t <= 0)
        t.comp_t = 1;
}

int build_plan(const pcdf_env *envs, int n_env, const pcdf_batch_tiles *tiles, pcdf_batch &B)
{
    using namespace pcdf;
    if (n_env < 1 || !envs)
        return fail(PCDF_EINVAL, "n_env must be >= 1 and envs non-NULL");
    B.tiles = tiles ? *tiles : pcdf_batch_tiles{0, 0, 0};
    default_tiles(B.tiles);
    if (B.tiles.row_rows > 4096 || B.tiles.dyn_slices > 512 || B.tiles.comp_t > PCDF_MAX_T)
        return fail(PCDF_EINVAL, "tile shape out of range");
    B.n_env = n_env;
    B.user.assign(envs, envs + n_env);
    B.plans.resize(n_env);
    B.desc.resize(n_env);
    B.off_bits.resize(n_env);
    B.off_carry.resize(n_env);
    B.off_mid.resize(n_env);
    B.off_static.resize(n_env);
    B.off_colmax.resize(n_env);
    B.off_dyn.resize(n_env);
    B.off_caps.resize(n_env);
    B.off_rep.resize(n_env);
    size_t off = 0, words = 0, words_comp = 0;
    std::vector<BatchItem> rows, dyn, ys, zs, comps;
    for (int e = 0; e < n_env; ++e) {
        const pcdf_env &U = envs[e];
        if (!U.occ || !U.comp_sq)
            return fail(PCDF_EINVAL, "environment %d: occ and comp_sq must be non-NULL", e);
        CompositePlan &p = B.plans[e];
        if (int rc = plan_composite(&U.grid, U.T, U.H, U.caps, p))
            return rc;
        if (p.S > 0 && !p.fused)
            return fail(PCDF_EINVAL, "environment %d: capsule stack bound %d too large for the batched kernel", e,
                        p.cap);
        const pcdf_grid &g = U.grid;
        const long long V = (long long)g.nx * g.ny * g.nz;
        const size_t nw = (size_t)g.nz * g.ny * ((g.nx + 31) / 32);
        B.off_bits[e] = off;
        off += align_up(nw * sizeof(uint32_t));
        B.off_carry[e] = off;
        off += align_up(nw * sizeof(uint2));
        B.off_mid[e] = off;
        off += align_up((size_t)V * 4);
        B.off_static[e] = off;
        off += align_up((size_t)V * 4);
        B.off_colmax[e] = off;
        off += align_up((size_t)g.nx * g.ny * 4);
        B.off_dyn[e] = off;
        off += align_up((size_t)p.slab * 4);
        B.off_caps[e] = off;
        off += align_up(p.ci.size() * sizeof(CapInfo));
        B.off_rep[e] = off;
        off += align_up(p.rep.size());
        words = std::max(words, smem_words_env(p, g, U.H));
        words_comp = std::max(words_comp, smem_words_comp(p));

        BatchEnv &D = B.desc[e];
        std::memset(&D, 0, sizeof(D));
        D.nx = g.nx;
        D.ny = g.ny;
        D.nz = g.nz;
        D.T = U.T;
        D.H = U.H;
        D.zlo = p.zlo;
        D.S = p.S;
        D.cap = p.cap;
        D.W = (g.nx + 31) / 32;
        D.vox = g.vox;
        const int nrows = g.ny * g.nz;
        for (int r = 0; r < nrows; r += B.tiles.row_rows)
            rows.push_back({kRow, e, r, 0});
        D.need[kRow] = (nrows + B.tiles.row_rows - 1) / B.tiles.row_rows;
        const int nxb = (g.nx + kThreads - 1) / kThreads;  // column blocks of a slice (<= 4)
        for (int t = 0; t < U.T; ++t)
            for (int s = 0; s < p.S; s += B.tiles.dyn_slices)
                for (int xb = 0; xb < nxb; ++xb)
                    dyn.push_back({kDyn, e, t, s * 16 + xb});
        D.need[kDyn] = U.T * ((p.S + B.tiles.dyn_slices - 1) / B.tiles.dyn_slices) * nxb;
        const long long zcols = (long long)g.nx * g.ny;
        for (int z = 0; z < g.nz; ++z)
            for (int w = 0; w < D.W; ++w)
                ys.push_back({kY, e, z, w});
        D.need[kY] = g.nz * D.W;
        for (long long c = 0; c < zcols; c += lean::kCols)
            zs.push_back({kZ, e, (int)c, 0});
        D.need[kZ] = (int)((zcols + lean::kCols - 1) / lean::kCols);
        // composite items t-fastest within a column block: the blocks of one
        // column range run together and share the static column in L2
        for (long long c = 0; c < zcols; c += kThreads)
            for (int t = 0; t < U.T; t += B.tiles.comp_t)
                comps.push_back({kComp, e, t, (int)c});
    }
    B.items.clear();
    for (auto *v : {&rows, &dyn, &ys, &zs})
        B.items.insert(B.items.end(), v->begin(), v->end());
    B.n_first = (int)B.items.size();
    B.items.insert(B.items.end(), comps.begin(), comps.end());
    B.off_desc = off;
    off += align_up(sizeof(BatchEnv) * n_env);
    B.off_items = off;
    off += align_up(sizeof(BatchItem) * B.items.size());
    B.off_state = off;
    off += align_up(sizeof(int) * (3 + 4 * (size_t)n_env));
    B.bytes = off;
    B.smem = words * 4;
    B.smem_comp = std::max<size_t>(words_comp * 4, 16);
    if (B.smem > 227 * 1024 || B.smem_comp > 227 * 1024)
        return fail(PCDF_EINVAL, "an environment needs %zu bytes of shared memory (limit 227 KB)",
                    std::max(B.smem, B.smem_comp));
    cudaError_t e = cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B.smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batched_comp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B.smem_comp);
    if (e != cudaSuccess)
        return cuda_fail(e, "batched kernel attributes");
    int dev = 0, sms = 0, per_sm = 0, per_sm_comp = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched, kThreads, B.smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_comp, k_batched_comp, kThreads, B.smem_comp);
    if (e != cudaSuccess)
        return cuda_fail(e, "batched kernel occupancy");
    B.blocks = std::max(1, sms * std::max(per_sm, 1));
    B.blocks_comp = std::max(1, sms * std::max(per_sm_comp, 1));
    return PCDF_OK;
}

}  // namespace

extern "C" {

int pcdf_batch_create(const pcdf_env *envs, int32_t n_env, const pcdf_batch_tiles *tiles, pcdf_batch **out)
{
    if (!out)
        return fail(PCDF_EINVAL, "out is NULL");
    *out = nullptr;
    pcdf_batch *B = new pcdf_batch();
    if (int rc = build_plan(envs, n_env, tiles, *B)) {
        delete B;
        return rc;
    }
    *out = B;
    return PCDF_OK;
}

void pcdf_batch_destroy(pcdf_batch *b) { delete b; }

int pcdf_batch_workspace_bytes(const pcdf_batch *b, size_t *bytes)
{
    if (!b || !bytes)
        return fail(PCDF_EINVAL, "batch and bytes must be non-NULL");
    *bytes = b->bytes;
    return PCDF_OK;
}

int pcdf_batch_tiles_used(const pcdf_batch *b, pcdf_batch_tiles *tiles)
{
    if (!b || !tiles)
        return fail(PCDF_EINVAL, "batch and tiles must be non-NULL");
    *tiles = b->tiles;
    return PCDF_OK;
}

int pcdf_batch_block_stage(pcdf_batch *b, int32_t env, int32_t stage)
{
    if (!b || env < 0 || env >= b->n_env || stage < 0 || stage > 2)
        return fail(PCDF_EINVAL, "batch, environment %d or stage %d out of range (stages 0 to 2 have waiters)", env,
                    stage);
    b->desc[env].need[stage] = 1 << 30;  // above any item count: the waits on it can only expire
    return PCDF_OK;
}

int pcdf_batch_upload(pcdf_batch *b, void *workspace, size_t workspace_bytes, void *stream)
{
    using namespace pcdf;
    if (!b || !workspace)
        return fail(PCDF_EINVAL, "batch and workspace must be non-NULL");
    if (!aligned(workspace, kAlign))
        return fail(PCDF_EINVAL, "workspace must be %zu-byte aligned", kAlign);
    if (workspace_bytes < b->bytes)
        return fail(PCDF_ENOMEM, "workspace %zu bytes < %zu needed", workspace_bytes, b->bytes);
    char *ws = (char *)workspace;
    cudaStream_t st = (cudaStream_t)stream;
    for (int e = 0; e < b->n_env; ++e) {
        BatchEnv &D = b->desc[e];
        D.occ = b->user[e].occ;
        D.comp_sq = b->user[e].comp_sq;
        D.bits = (uint32_t *)(ws + b->off_bits[e]);
        D.carry = (uint2 *)(ws + b->off_carry[e]);
        D.mid = (int32_t *)(ws + b->off_mid[e]);
        D.static_sq = (int32_t *)(ws + b->off_static[e]);
        D.colmax = (int32_t *)(ws + b->off_colmax[e]);
        D.vec = ((long long)D.nx * D.ny) % 4 == 0 && ((uintptr_t)D.comp_sq & 15u) == 0 &&
                ((uintptr_t)D.static_sq & 15u) == 0;
        D.dyn = (int32_t *)(ws + b->off_dyn[e]);
        D.caps = (const CapInfo *)(ws + b->off_caps[e]);
        const std::vector<uint8_t> &rp = b->plans[e].rep;
        D.rep = rp.empty() ? nullptr : (const uint8_t *)(ws + b->off_rep[e]);
        if (!rp.empty()) {
            cudaError_t err = cudaMemcpyAsync(ws + b->off_rep[e], rp.data(), rp.size(), cudaMemcpyHostToDevice, st);
            if (err != cudaSuccess)
                return cuda_fail(err, "batch upload");
        }
        const std::vector<CapInfo> &ci = b->plans[e].ci;
        if (!ci.empty()) {
            cudaError_t err = cudaMemcpyAsync(ws + b->off_caps[e], ci.data(), ci.size() * sizeof(CapInfo),
                                              cudaMemcpyHostToDevice, st);
            if (err != cudaSuccess)
                return cuda_fail(err, "batch upload");
        }
    }
    cudaError_t err = cudaMemcpyAsync(ws + b->off_desc, b->desc.data(), sizeof(BatchEnv) * b->n_env,
                                      cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(ws + b->off_items, b->items.data(), sizeof(BatchItem) * b->items.size(),
                              cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess)
        return cuda_fail(err, "batch upload");
    return PCDF_OK;
}

int pcdf_batch_run(const pcdf_batch *b, void *workspace, void *stream)
{
    using namespace pcdf;
    if (!b || !workspace)
        return fail(PCDF_EINVAL, "batch and workspace must be non-NULL");
    char *ws = (char *)workspace;
    cudaStream_t st = (cudaStream_t)stream;
    int *state = (int *)(ws + b->off_state);
    cudaError_t err = cudaMemsetAsync(state, 0, sizeof(int) * (3 + 4 * (size_t)b->n_env), st);
    if (err != cudaSuccess)
        return cuda_fail(err, "batch counter reset");
    const BatchEnv *desc = (const BatchEnv *)(ws + b->off_desc);
    const BatchItem *items = (const BatchItem *)(ws + b->off_items);
    k_batched<<<b->blocks, kThreads, b->smem, st>>>(desc, items, b->n_first, state, b->tiles.row_rows,
                                                   b->tiles.dyn_slices, b->tiles.comp_t);
    err = cudaGetLastError();
    if (err != cudaSuccess)
        return cuda_fail(err, "batched launch");
    const int n_comp = (int)b->items.size() - b->n_first;
    k_batched_comp<<<b->blocks_comp, kThreads, b->smem_comp, st>>>(desc, items + b->n_first, n_comp, state + 1,
                                                                   state + 2 + 4 * b->n_env, b->tiles.comp_t);
    err = cudaGetLastError();
    return err == cudaSuccess ? PCDF_OK : cuda_fail(err, "batched composite launch");
}

int pcdf_batch_error(const pcdf_batch *b, const void *workspace, void *stream, int32_t *code)
{
    if (!b || !workspace || !code)
        return fail(PCDF_EINVAL, "batch, workspace and code must be non-NULL");
    int word = 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t err = cudaMemcpyAsync(&word, (const char *)workspace + b->off_state + sizeof(int), sizeof(int),
                                      cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess)
        err = cudaStreamSynchronize(st);
    if (err != cudaSuccess)
        return cuda_fail(err, "batch error read");
    *code = word ? PCDF_ETIMEOUT : PCDF_OK;
    return PCDF_OK;
}

int pcdf_batch_autotune_workspace_bytes(const pcdf_env *envs, int32_t n_env, size_t *bytes)
{
    if (!bytes)
        return fail(PCDF_EINVAL, "bytes is NULL");
    // the smallest tiles give the longest item list, hence the largest layout
    pcdf_batch_tiles t{8, 1, 1};
    pcdf_batch B;
    if (int rc = build_plan(envs, n_env, &t, B))
        return rc;
    *bytes = B.bytes;
    return PCDF_OK;
}

int pcdf_batch_autotune(const pcdf_env *envs, int32_t n_env, void *workspace, size_t workspace_bytes, void *stream,
                        int32_t reps, pcdf_batch_tiles *best, float *best_ms)
{
    if (!best)
        return fail(PCDF_EINVAL, "best is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(PCDF_ECUDA, "event creation failed");
    float best_t = -1.f;
    int rc = PCDF_OK;
    for (int rr : {8, 32, 128})
        for (int ds : {1, 4})
            for (int ct : {1, 4}) {
                pcdf_batch_tiles t{rr, ds, ct};
                pcdf_batch B;
                if ((rc = build_plan(envs, n_env, &t, B)))
                    goto done;
                if ((rc = pcdf_batch_upload(&B, workspace, workspace_bytes, stream)))
                    goto done;
                if ((rc = pcdf_batch_run(&B, workspace, stream)))  // warm-up
                    goto done;
                float tot = 0.f;
                for (int k = 0; k < std::max(reps, 1); ++k) {
                    cudaEventRecord(e0, st);
                    if ((rc = pcdf_batch_run(&B, workspace, stream)))
                        goto done;
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess) {
                        rc = fail(PCDF_ECUDA, "autotune synchronisation failed");
                        goto done;
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    tot += ms;
                }
                int32_t code = 0;
                if ((rc = pcdf_batch_error(&B, workspace, stream, &code)))
                    goto done;
                if (code != PCDF_OK) {
                    rc = fail(code, "batched kernel reported a dependency timeout during autotuning");
                    goto done;
                }
                tot /= std::max(reps, 1);
                if (best_t < 0.f || tot < best_t) {
                    best_t = tot;
                    *best = t;
                }
            }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == PCDF_OK && best_ms)
        *best_ms = best_t;
    return rc;
}

}  // extern "C"
