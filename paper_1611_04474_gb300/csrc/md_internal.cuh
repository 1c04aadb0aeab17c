// md_internal.cuh -- shared device helpers and the workspace layout of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "md_nonbonded.h"

namespace mdnb {

// (kcal/mol/A)/amu expressed in A/fs^2
constexpr double kAccelPerForcePerMass = 4.184e-4;
// fixed-point scale of MD_ACCUM_FIXED64: one unit is 2^-32 kcal/mol/A
constexpr float kFixedScale = 4294967296.0f;
// |term| must stay below 2^31 so that term * 2^32 fits an int64
constexpr float kFixedLimit = 2147483648.0f;

constexpr int kMaxTypes = 32;

// Modes whose forces are int64 at 2^-32 (accumulators u64[3][n], output int64[n][3]).
__host__ __device__ constexpr bool fixed_output(int mode)
{
    return mode == MD_ACCUM_FIXED64 || mode == MD_ACCUM_FIXED_TILE;
}

// Per-block partial results of a force or kinetic-energy pass, reduced later in a
// fixed order so that sums do not depend on block scheduling.
struct Partial {
    double e_lj, e_c, w;
    unsigned long long count;
};

// Host-side description of the periodic box in the forms the kernels use.
struct BoxF {
    double L[3];
    float Lhi[3];   // float(L): the leading part of L
    float Llo[3];   // float(L - Lhi): the remainder, so Lhi + Llo == L to ~2^-48 L
    float invL[3];  // 1/L rounded to float
    double inv_edge[3];  // dims / L (one IEEE division, the same bits on host and device)
    float Lin[3];        // the largest float <= L: x in [0, Lin) means (double)x in [0, L)
    float inv_edge_f[3]; // inv_edge rounded to float
    int dims[3];
    int ncell;
};

BoxF make_box(const double *L, const int32_t *dims);

// One system of a batch as the kernels see it (device array in the batch workspace).
struct SysDesc {
    BoxF box;
    const float2 *AB;
    int ntypes;
    float kc;
    double kc64;
    float rc2, rc2m;   // exact cutoff test, conservative filter threshold
    int atom_offset;   // first atom (input order and sorted order alike)
    int natoms;
    int cell_offset;   // first global cell
    int mi;            // some axis has two cells: per-pair minimum image
};


struct WsLayout {
    size_t cell_id;     // int32 [n]          cell of each input atom
    size_t cell_cnt;    // int32 [ncell + 1]  per-cell counts, then scatter cursors; the last
                        //                    counts the finished blocks of the step's build pass
    size_t perm_tmp;    // int32 [n]          unsorted slot -> input index
    size_t accum;       // 32 B x n           sorted-order force accumulators
    size_t partials;    // Partial [nslots]
    size_t ev;          // double[4]          energy/virial scratch of md_step
    size_t st_cell_start, st_perm, st_pos_q_sorted, st_type_sorted, st_pos_q;  // md_step only
    size_t clu_pos_q, clu_type, clu_order;  // cluster-pair kernel: per-cell reordered copies
    size_t clu_box;     // float4 [2 n]  cluster boxes: lo at the cluster's first slot, hi at n + it
    size_t work;        // int[2] item counters of persistent force launches
    size_t bins;        // int32 [ncell][bin_cap] members of each cell by arrival (MD step)
    size_t v_ref;       // float4 [n]  positions at the last cell rebuild (Verlet step only)
    size_t v_flags;     // VerletFlags (Verlet step only)
    size_t total;
    int nslots;
    int bin_cap;        // 0: no bins (the step scatters through perm_tmp)
};

// CTAs that share one cell pair of the cluster-pair kernel in boxes with an axis of 2
// cells (their few cell pairs are long), each taking every kMiSplit-th home cluster.
constexpr int kMiSplit = 4;

// Members per cell that the MD step's bins hold: twice the mean occupancy plus 64,
// rounded up to 32.  A cell with more members is gathered by a scan of the cell ids.
int bin_capacity(int n, int ncell);
// split: the box has an axis of 2 cells (its cluster-pair CTAs are split kMiSplit ways,
// each with a partial); the default reserves for that case
WsLayout ws_layout(int n, int ncell, bool bins = true, bool verlet = false, bool split = true);

// Device state of the Verlet step (md_step_verlet), in its workspace.
struct VerletFlags {
    int rebuild;             // the cells of this step are rebuilt (1) or kept (0)
    unsigned maxdisp2;       // bits of the largest squared move since the rebuild (a float)
};

// Layout of the batch workspace (byte offsets), derived on the host from the systems.
struct BatchLayout {
    int nsys, n, ncell, ncell_mi, ncell_reg;
    size_t sys;         // SysDesc [nsys]
    size_t cell_sys;    // int [ncell]: system of each global cell
    size_t cell_list;   // int [ncell]: regular systems' cells, then minimum-image ones
    size_t atom_sys;    // int [n]: system of each atom
    WsLayout run;       // the per-run scratch of the single-system path, sized for n, ncell
    size_t run_base;    // where that scratch starts
    size_t total;
};

// ------------------------------------------------- programmatic dependent launch
// The MD step's kernels after the first are launched with programmatic stream
// serialization: such a kernel may be scheduled while its predecessor finishes, and
// waits (pdl_wait) for the predecessor's completion and memory before it touches any
// data that an earlier launch writes.  A kernel lets its dependent be scheduled
// (pdl_trigger) once it has started.  Launched the ordinary way, both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t stream, Args &&...args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ----------------------------------------------------------------- device helpers

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t bits)
{
    if (status) atomicOr(status, bits);
}

// 0 <= x < L for a finite L > 0, decided on the bit patterns (non-negative doubles
// order like their bits), which keeps the test off the FP64 pipe.  -0.0 is inside, as
// for the floating-point comparison; NaN and infinities are not.
__device__ __forceinline__ bool in_box_f64(double x, double L)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned long long a = u & 0x7fffffffffffffffull;
    return (u == a || a == 0ull) && a < (unsigned long long)__double_as_longlong(L);
}

// Wrap a coordinate into [0, L) in FP64 (the documented rule).  A coordinate already
// in [0, L) is returned as it is, which is what the rule gives for it (even when x/L
// rounds up to 1, the fold-back restores x exactly), without the FP64 division.
__device__ __forceinline__ double wrap_coord(double x, double L)
{
    if (in_box_f64(x, L)) return x;
    double w = x - L * floor(x / L);
    if (w < 0.0) w += L;
    if (w >= L) w -= L;
    return w;
}

// Cell index along one axis of a wrapped coordinate: floor(w * (n/L)) clamped, with
// inv_edge = n/L from the host.
__device__ __forceinline__ int cell_coord(double w, int nc, double inv_edge)
{
    double f = floor(w * inv_edge);
    return f < 0.0 ? 0 : (f > (double)(nc - 1) ? nc - 1 : (int)f);
}

__device__ __forceinline__ bool finite3(double x, double y, double z)
{
    return isfinite(x) && isfinite(y) && isfinite(z);
}

// Cell index along axis k of a float coordinate, equal to
// cell_coord(wrap_coord((double)x, L), ...) for every x.  For x in [0, Lin) the FP32
// product t = x * (n/L) decides unless it lies within 2.5e-7 t of an integer: the FP32
// and FP64 products differ by less than 1.2e-7 t (two float roundings, of n/L and of
// the product), so outside that band both have the same floor.  Inside it, and for x
// outside [0, Lin), the FP64 rule runs.
__device__ __forceinline__ int cell_coord_fast(float x, const BoxF &box, int k)
{
    if (x >= 0.0f && x < box.Lin[k]) {
        const float t = __fmul_rn(x, box.inv_edge_f[k]);
        const float fl = floorf(t);
        const float fr = __fsub_rn(t, fl);  // exact (Sterbenz for t >= 1; fl = 0 below)
        const float tol = __fmul_rn(t, 2.5e-7f);
        if (fr > tol && fr < __fsub_rn(1.0f, tol)) {
            const int c = (int)fl;
            return c < box.dims[k] ? c : box.dims[k] - 1;
        }
    }
    return cell_coord(wrap_coord((double)x, box.L[k]), box.dims[k], box.inv_edge[k]);
}

// Cell of a float position under the documented rule (FP64 wrap of the float value,
// floor(w * n/L) clamped); a non-finite coordinate sets the status and gives cell 0.
__device__ __forceinline__ int cell_of(const float4 &p, const BoxF &box, uint32_t *status)
{
    if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z))) {
        set_status(status, MD_STATUS_NONFINITE);
        return 0;
    }
    const int cx = cell_coord_fast(p.x, box, 0);
    const int cy = cell_coord_fast(p.y, box, 1);
    const int cz = cell_coord_fast(p.z, box, 2);
    return cx + box.dims[0] * (cy + box.dims[1] * cz);
}

// Velocity-Verlet updates with every rounding spelled out, in the oracle's order: the
// per-atom factor c = ((dt/2) (1/m)) 4.184e-4, then v + F c and x + dt v each as one
// fused multiply-add (one rounding).  Every kernel that moves atoms uses these, so the
// single-system and batched steps agree bit for bit.
__device__ __forceinline__ double kick_factor(double im, double half_dt)
{
    return __dmul_rn(__dmul_rn(half_dt, im), kAccelPerForcePerMass);
}
__device__ __forceinline__ double kick_velocity(double v, double f, double c)
{
    return __fma_rn(f, c, v);
}
__device__ __forceinline__ double drift_coord(double x, double v, double dt)
{
    return __fma_rn(dt, v, x);
}

// A float position wrapped into the box by the FP64 rule and rounded back to float
// (non-finite coordinates give the origin); the charge is kept.  A coordinate in
// [0, Lin) wraps to itself, so the FP64 work runs only for the rare others.
__device__ __forceinline__ float4 wrap_pos_f(const float4 &p, const BoxF &box)
{
    float4 o = p;
    if (!(p.x >= 0.0f && p.x < box.Lin[0] && p.y >= 0.0f && p.y < box.Lin[1] && p.z >= 0.0f &&
          p.z < box.Lin[2])) {
        const double x = p.x, y = p.y, z = p.z;
        if (isfinite(x) && isfinite(y) && isfinite(z)) {
            o.x = (float)wrap_coord(x, box.L[0]);
            o.y = (float)wrap_coord(y, box.L[1]);
            o.z = (float)wrap_coord(z, box.L[2]);
        } else {
            o.x = o.y = o.z = 0.0f;
        }
    }
    return o;
}

// Sorted-order slot of one atom: its input index, its wrapped float position and
// charge, its type (the outputs of the cell build).
__device__ __forceinline__ void place(int e, int slot, const float4 *__restrict__ pos_q,
                                      const int32_t *__restrict__ type, const BoxF &box,
                                      int32_t *__restrict__ perm, float4 *__restrict__ pos_q_sorted,
                                      int32_t *__restrict__ type_sorted)
{
    perm[slot] = e;
    pos_q_sorted[slot] = wrap_pos_f(pos_q[e], box);
    type_sorted[slot] = type[e];
}

// Force on atom i as FP64 from the forces array of a mode (input order).
__device__ __forceinline__ void load_force(const void *forces, int mode, int i, double f[3])
{
    if (mode == MD_ACCUM_F32) {
        const float *F = static_cast<const float *>(forces);
        f[0] = F[3 * i];
        f[1] = F[3 * i + 1];
        f[2] = F[3 * i + 2];
    } else if (fixed_output(mode)) {
        const long long *F = static_cast<const long long *>(forces);
        const double s = 1.0 / 4294967296.0;
        f[0] = (double)F[3 * i] * s;
        f[1] = (double)F[3 * i + 1] * s;
        f[2] = (double)F[3 * i + 2] * s;
    } else {
        const double *F = static_cast<const double *>(forces);
        f[0] = F[3 * i];
        f[1] = F[3 * i + 1];
        f[2] = F[3 * i + 2];
    }
}

// Minimum-image displacement xi - xj along one axis in FP32 for coordinates in
// [0, L].  The image is chosen from the rounded difference, then the difference is
// formed again so that it is exact up to one rounding of the result: the box shift
// Lhi is subtracted from the coordinate near L (exact by Sterbenz), and the
// remainder Llo is applied last.
__device__ __forceinline__ float min_image_f32(float xi, float xj, float Lhi, float Llo, float invL)
{
    const float d0 = __fsub_rn(xi, xj);
    const float k = rintf(__fmul_rn(d0, invL));
    const float a = __fsub_rn(xi, k > 0.0f ? Lhi : 0.0f);
    const float b = __fsub_rn(xj, k < 0.0f ? Lhi : 0.0f);
    return __fsub_rn(__fsub_rn(a, b), __fmul_rn(k, Llo));
}

__device__ __forceinline__ double min_image_f64(double xi, double xj, double L)
{
    double d = xi - xj;
    return d - L * rint(d / L);
}

// Pair arithmetic of Eq. 1 + Eq. 2 in FP32 with every rounding spelled out, so that
// every kernel produces the same bits for the same pair (no compiler contraction).
__device__ __forceinline__ float pair_r2(float dx, float dy, float dz)
{
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// 1/sqrt(x) from the hardware approximation (MUFU; relative error near 2^-22, well
// inside the 1e-5 force criterion, so no refinement step).
__device__ __forceinline__ float rsqrt_hw(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Scalar f of F = f * r (Eq. 1: A/r^14 - B/r^8 = (A r^-6 - B) r^-8, Eq. 2:
// k q1 q2 / r^3); also returns 1/r, 1/r^2, 1/r^6 for the energies.  The Coulomb term
// joins the LJ term in one fused multiply-add, so that no separate multiply feeds an
// add (which a compiler could fuse in one kernel and not in another).
__device__ __forceinline__ float pair_f(float r2, float A, float B, float kqq, float &ir,
                                        float &ir2, float &ir6)
{
    ir = rsqrt_hw(r2);
    ir2 = __fmul_rn(ir, ir);
    ir6 = __fmul_rn(__fmul_rn(ir2, ir2), ir2);
    const float ir8 = __fmul_rn(ir6, ir2);
    const float lj = __fmul_rn(ir8, __fmaf_rn(A, ir6, -B));
    return __fmaf_rn(__fmul_rn(kqq, ir2), ir, lj);
}

__device__ __forceinline__ float pair_u_lj(float A, float B, float ir6)
{
    return __fmaf_rn(A * (1.0f / 12.0f), __fmul_rn(ir6, ir6), -__fmul_rn(B * (1.0f / 6.0f), ir6));
}

// Round one pair-force component to the MD_ACCUM_FIXED64 grid (2^-32 kcal/mol/A),
// round-to-nearest-even; flags terms that do not fit and contributes nothing for them.
__device__ __forceinline__ long long to_fixed(float v, uint32_t *status)
{
    if (!(fabsf(v) < kFixedLimit)) {
        set_status(status, isfinite(v) ? MD_STATUS_FIXED_OVERFLOW : MD_STATUS_NONFINITE);
        return 0;
    }
    return __float2ll_rn(v * kFixedScale);
}

__device__ __forceinline__ int clamp_type(int t, int ntypes, uint32_t *status)
{
    if ((unsigned)t >= (unsigned)ntypes) {
        set_status(status, MD_STATUS_BAD_TYPE);
        return 0;
    }
    return t;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Bounding boxes of the clusters (8 consecutive slots) of one cell of m atoms in its final
// order, p pointing at its first atom (which is slot s0): lo at box[first slot], hi at
// box[n + first slot]; the last cluster's empty slots are left out.  The cell's atoms
// must have been written before (the caller synchronises its block first).
template <int NT>
__device__ __forceinline__ void write_cluster_boxes(const float4 *p, int s0, int m, float4 *box, int n)
{
    for (int k = threadIdx.x; 8 * k < m; k += NT) {
        const int b = s0 + 8 * k, e = min(m - 8 * k, 8);
        const float4 *c = p + 8 * k;
        float4 lo = c[0], hi = lo;
        for (int t = 1; t < e; ++t) {
            const float4 q = c[t];
            lo.x = fminf(lo.x, q.x); hi.x = fmaxf(hi.x, q.x);
            lo.y = fminf(lo.y, q.y); hi.y = fmaxf(hi.y, q.y);
            lo.z = fminf(lo.z, q.z); hi.z = fmaxf(hi.z, q.z);
        }
        box[b] = lo;
        box[(size_t)n + b] = hi;
    }
}

// Sum (e_lj, e_c, w, count) over the block into *slot in a fixed order.
template <int kThreads>
__device__ __forceinline__ void block_partial_to(double e_lj, double e_c, double w,
                                                 unsigned long long cnt, Partial *slot)
{
    __shared__ double s_e[3][kThreads / 32];
    __shared__ unsigned long long s_c[kThreads / 32];
    e_lj = warp_sum(e_lj);
    e_c = warp_sum(e_c);
    w = warp_sum(w);
    cnt = warp_sum(cnt);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_e[0][warp] = e_lj;
        s_e[1][warp] = e_c;
        s_e[2][warp] = w;
        s_c[warp] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Partial p = {0.0, 0.0, 0.0, 0ull};
        for (int k = 0; k < kThreads / 32; ++k) {
            p.e_lj += s_e[0][k];
            p.e_c += s_e[1][k];
            p.w += s_e[2][k];
            p.count += s_c[k];
        }
        *slot = p;
    }
}

// The same into partials[blockIdx.x].
template <int kThreads>
__device__ __forceinline__ void block_partial(double e_lj, double e_c, double w,
                                              unsigned long long cnt, Partial *partials)
{
    block_partial_to<kThreads>(e_lj, e_c, w, cnt, partials + blockIdx.x);
}

}  // namespace mdnb

// Launchers implemented in the .cu files (all enqueue on `stream`, return cudaError_t).
namespace mdnb {
cudaError_t launch_build_cells(const float4 *pos_q, const int32_t *type, int n, const BoxF &box,
                               int32_t *cell_start, int32_t *perm, float4 *pos_q_sorted,
                               int32_t *type_sorted, const WsLayout &ws, char *wsp,
                               uint32_t *status, cudaStream_t stream);

struct ForceArgs {
    const int32_t *cell_start;
    const int32_t *perm;
    const float4 *pos_q_sorted;
    const int32_t *type_sorted;
    int n;
    BoxF box;
    const float2 *AB;
    int ntypes;
    float k_coulomb;
    double k_coulomb64;
    float rc;
    double rc64;
    int mode;
    int algo;
    void *forces_out;
    double *energy_virial_out;
    unsigned long long *pair_count_out;
    uint32_t *status;
    // within-cell order already the cluster kernel's (from the fused MD-step build):
    // no ordering pass, perm maps each slot to its input index
    int presorted = 0;
    // the build pass of the MD step already zeroed the cluster-order accumulators (and
    // the persistent launches' item counters)
    int accum_zeroed = 0;
    // bounding boxes of the presorted cells' clusters (lo at the first slot of a cluster, hi
    // at n + that slot), written by the MD step's build; null where none were written
    const float4 *clu_box = nullptr;
    // Verlet step: the cells (cell_start, perm, type_sorted) are those of the last rebuild
    // and the current positions come from this input-order float copy through perm
    const float4 *gather_pq = nullptr;
    // optional half kick v += dt/2 a(F) applied as the forces are written (MD step)
    double *kick_vel = nullptr;
    const float *kick_inv_mass = nullptr;
    double kick_half_dt = 0.0;
};

cudaError_t launch_forces(const ForceArgs &a, const WsLayout &ws, char *wsp, cudaStream_t stream);
int half_shell_pairs_per_cell(const BoxF &box);
void cutoff_thresholds(const BoxF &box, double rc, bool mi, float *rc2, float *rc2m);
cudaError_t launch_half_shell(const ForceArgs &a, const WsLayout &ws, char *wsp, Partial *partials,
                              int *nblocks_out, cudaStream_t stream);
cudaError_t launch_finalize_cluster(const ForceArgs &a, const void *accum, const WsLayout &ws,
                                    char *wsp, int n, cudaStream_t stream);
cudaError_t launch_cluster(const ForceArgs &a, const WsLayout &ws, char *wsp, Partial *partials,
                           int *nblocks_out, cudaStream_t stream);

// Batched forms: every system of the batch in one launch per kernel.
struct BatchArgs {
    const SysDesc *sys;
    const int *cell_sys;
    const int *cell_list;
    const int *atom_sys;
    int nsys, n, ncell, ncell_mi, ncell_reg;
    int max_ntypes;  // largest LJ table of the batch: sizes the kernels' shared copy
};
cudaError_t launch_cluster_batched(int mode, bool mi, const BatchArgs &b, const int32_t *cell_start,
                                   const float4 *pq, const int32_t *ty, void *accum,
                                   Partial *partials, uint32_t *status,
                                   unsigned long long *sys_pair_count, int *persist_work,
                                   cudaStream_t stream);
cudaError_t launch_kick_drift_build(double *pos, double *vel, const void *forces, int mode,
                                    const float *inv_mass, const float *q, const int32_t *type, int n,
                                    const BoxF &box_in, const BatchArgs *b, double dt, double half_dt,
                                    bool kick, float4 *pos_q, int32_t *cell_start, int32_t *perm,
                                    float4 *pos_q_sorted, int32_t *type_sorted, const WsLayout &ws,
                                    char *wsp, uint32_t *status, cudaStream_t stream);
cudaError_t launch_forces_batched(const ForceArgs &a, const BatchArgs &b,
                                  unsigned long long *sys_pair_count, const WsLayout &ws,
                                  char *wsp, cudaStream_t stream, int shape_reg, int shape_mi);

cudaError_t launch_kick(double *vel, const void *forces, int mode, const float *inv_mass, int n,
                        double half_dt, cudaStream_t stream);

// Verlet step passes (md_verlet.cu and md_cells.cu).
cudaError_t launch_verlet_drift(double *pos, double *vel, const void *forces, int mode,
                                const float *inv_mass, const float *q, int n, const BoxF &box,
                                double dt, double half_dt, bool kick, float4 *pos_q,
                                const float4 *x_ref, void *accum, VerletFlags *flags,
                                uint32_t *status, cudaStream_t stream);
cudaError_t launch_verlet_decide(VerletFlags *flags, float threshold2, bool force,
                                 unsigned long long *rebuilds, cudaStream_t stream);
cudaError_t launch_verlet_rebuild(const float4 *pos_q, const int32_t *type, int n, const BoxF &box,
                                  int32_t *cell_start, int32_t *perm, float4 *pos_q_sorted,
                                  int32_t *type_sorted, float4 *x_ref, const int *run_flag,
                                  const WsLayout &ws, char *wsp, uint32_t *status,
                                  cudaStream_t stream);
cudaError_t launch_energy_log_row(const double *vel, const float *inv_mass, int n,
                                  const double *energy_virial, double *row, const WsLayout &ws,
                                  char *wsp, cudaStream_t stream);
}  // namespace mdnb
