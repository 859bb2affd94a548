// Host-side helpers shared by the C ABI entry points (plan.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "pcdf_internal.cuh"

namespace pcdf {
namespace host {

constexpr size_t kAlign = 256;

const char *last_error();
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *where);
size_t align_up(size_t x);
int check_grid(const pcdf_grid *g);
long long nvox(const pcdf_grid *g);
long long floordiv(long long a, long long b);
int make_capinfo(const pcdf_grid *g, int T, int H, const int32_t *caps, std::vector<CapInfo> &out, int *zlo,
                 int *zhi);
int check_caps_args(int T, int H, const int32_t *caps);
bool aligned(const void *p, size_t a);
int run_full_edt(const pcdf_grid *g, int mode, const uint8_t *occ, const CapBatch *caps, int H, int32_t *sq,
                 float *sdf, void *ws, cudaStream_t st, int32_t *colmax = nullptr);
size_t full_edt_ws(const pcdf_grid *g);

// Slab geometry and capsule table of one composite request.
struct CompositePlan {
    std::vector<CapInfo> ci;
    int zlo = 0, zhi = -1, S = 0;
    long long slab = 0;  // T * S * nx * ny
    bool fused = false;  // analytic x+y kernel (else row pass + y envelope)
    int cap = 0;         // its per-thread stack capacity
    size_t need = 0;     // workspace bytes
    size_t colmax_off = 0;  // workspace offset of the static column maxima
    std::vector<uint8_t> rep;  // [T][S] first slab slice with the same capsule cross-sections (empty: identity)
};

// the slab map of a plan as a kernel parameter (identity when the plan has none)
void slab_map(const CompositePlan &p, SlabMap &m);

int plan_composite(const pcdf_grid *grid, int T, int H, const int32_t *caps, CompositePlan &p);
int32_t *plan_mid(const CompositePlan &p, void *workspace);
int check_ws(const CompositePlan &p, void *workspace, size_t workspace_bytes);
int composite_prepare(const pcdf_grid *grid, int T, int H, const CompositePlan &p, void *workspace,
                      cudaStream_t st);
// fields t = t0 .. t0 + nt - 1 (outputs indexed by the absolute t);
// have_colmax: the static column maxima are already at p.colmax_off in the
// workspace (written by the static build), so they are not recomputed
int composite_finish(const pcdf_grid *grid, const int32_t *static_sq, const float *static_sdf, int t0, int nt,
                     const CompositePlan &p, int32_t *comp_sq, float *comp_sdf, void *workspace, cudaStream_t st,
                     bool have_colmax = false);

}  // namespace host
}  // namespace pcdf
