// md_cells.cu -- cell binning by counting sort (Section II.A cell-list method; the
// per-cell arrays of Section II.B item 2 instead of linked lists).
//
//   1. k_cell_index : wrap each coordinate in FP64, cell index, per-cell histogram
//   2. k_scan_cells : exclusive scan of the histogram -> cell_start, scatter cursors
//   3. k_scatter    : each atom takes a slot of its cell (atomic cursor; order within
//                     a cell is arbitrary here)
//   4. k_cell_sort  : one block per cell ranks its members by input index, which
//                     restores a deterministic order, and gathers the wrapped
//                     float4 positions and types into sorted order.
#include "md_internal.cuh"

namespace mdnb {
namespace {

constexpr int kIndexThreads = 1024;  // atoms per block of the counting passes
constexpr int kStepThreads = 256;    // atoms per block of the fused MD-step pass (FP64 work)
constexpr int kStepSmemCells = 4 * kStepThreads;  // per-block shared histogram up to this
constexpr int kSmemCells = 8192;     // per-block shared histogram up to this many cells
constexpr int kScanThreads = 1024;
constexpr int kSortThreads = 128;
constexpr int kSortChunk = 2048;  // members staged in shared memory at a time

// Per-block histogram in shared memory (grids with up to kSmemCells cells), then one
// global add per touched cell; larger grids count with warp-aggregated global atomics.
template <bool SMEM>
__global__ void __launch_bounds__(kIndexThreads)
k_cell_index(const float4 *__restrict__ pos_q, int n, BoxF box, int *__restrict__ cell_id,
             int *__restrict__ cell_cnt, uint32_t *status)
{
    extern __shared__ int s_hist[];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int ncell = box.ncell;
    if (SMEM) {
        for (int t = threadIdx.x; t < ncell; t += blockDim.x) s_hist[t] = 0;
        __syncthreads();
    }
    int c = -1;
    if (i < n) {
        c = cell_of(pos_q[i], box, status);
        cell_id[i] = c;
    }
    if (SMEM) {
        // one shared atomic per distinct cell of the warp (consecutive atoms often share
        // a cell)
        const unsigned act = __ballot_sync(0xffffffffu, c >= 0);
        const unsigned grp = __match_any_sync(0xffffffffu, c) & act;
        if (c >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&s_hist[c], __popc(grp));
        __syncthreads();
        for (int t = threadIdx.x; t < ncell; t += blockDim.x)
            if (s_hist[t]) atomicAdd(&cell_cnt[t], s_hist[t]);
    } else {
        const unsigned act = __ballot_sync(0xffffffffu, c >= 0);
        const unsigned grp = __match_any_sync(0xffffffffu, c) & act;
        if (c >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&cell_cnt[c], __popc(grp));
    }
}

// Single block: exclusive scan of the per-cell counts.  Writes cell_start[0..ncell]
// and turns the counts into scatter cursors (= cell_start[c]).
__global__ void __launch_bounds__(kScanThreads)
k_scan_cells(int *__restrict__ cnt_cursor, int ncell, int *__restrict__ cell_start)
{
    __shared__ int sums[kScanThreads];
    int t = threadIdx.x;
    int per = (ncell + kScanThreads - 1) / kScanThreads;
    int lo = min(t * per, ncell), hi = min(lo + per, ncell);
    int s = 0;
    for (int c = lo; c < hi; ++c) s += cnt_cursor[c];
    sums[t] = s;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        int v = t >= off ? sums[t - off] : 0;
        __syncthreads();
        sums[t] += v;
        __syncthreads();
    }
    int run = sums[t] - s;
    for (int c = lo; c < hi; ++c) {
        int k = cnt_cursor[c];
        cell_start[c] = run;
        cnt_cursor[c] = run;
        run += k;
    }
    if (t == kScanThreads - 1) cell_start[ncell] = sums[t];
}

// Each atom takes a slot of its cell; the atoms of a warp that share a cell take
// consecutive slots with one atomic (the order is fixed later by k_cell_sort).
__global__ void __launch_bounds__(kIndexThreads)
k_scatter(const int *__restrict__ cell_id, int n, int *__restrict__ cursor, int *__restrict__ perm_tmp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int c = i < n ? cell_id[i] : -1;
    const unsigned act = __ballot_sync(0xffffffffu, c >= 0);
    const unsigned grp = __match_any_sync(0xffffffffu, c) & act;
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (c >= 0 && lane == leader) base = atomicAdd(&cursor[c], __popc(grp));
    base = __shfl_sync(0xffffffffu, base, leader < 0 ? 0 : leader);
    if (c >= 0) perm_tmp[base + __popc(grp & ((1u << lane) - 1u))] = i;
}

// One block per cell.  Members are distinct input indices, so the rank of a member
// among them (number of smaller members) is its slot in ascending input order.  Each
// thread ranks one member per round against the whole cell, staged in shared memory
// (in chunks for cells larger than kSortChunk).
__global__ void __launch_bounds__(kSortThreads)
k_cell_sort(const int *__restrict__ cell_start, const int *__restrict__ perm_tmp,
            const float4 *__restrict__ pos_q, const int32_t *__restrict__ type, BoxF box,
            int32_t *__restrict__ perm, float4 *__restrict__ pos_q_sorted,
            int32_t *__restrict__ type_sorted)
{
    __shared__ int chunk[kSortChunk];
    const int c = blockIdx.x;
    const int s0 = cell_start[c];
    const int m = cell_start[c + 1] - s0;
    if (m == 0) return;
    if (m <= kSortChunk) {
        for (int u = threadIdx.x; u < m; u += kSortThreads) chunk[u] = perm_tmp[s0 + u];
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += kSortThreads) {
            const int e = chunk[t];
            int rank = 0;
            for (int u = 0; u < m; ++u) rank += chunk[u] < e;
            place(e, s0 + rank, pos_q, type, box, perm, pos_q_sorted, type_sorted);
        }
        return;
    }
    for (int base = 0; base < m; base += kSortThreads) {
        const int t = base + threadIdx.x;
        const int e = t < m ? perm_tmp[s0 + t] : -1;
        int rank = 0;
        for (int c0 = 0; c0 < m; c0 += kSortChunk) {
            const int len = min(kSortChunk, m - c0);
            __syncthreads();
            for (int u = threadIdx.x; u < len; u += kSortThreads) chunk[u] = perm_tmp[s0 + c0 + u];
            __syncthreads();
            for (int u = 0; u < len; ++u) rank += chunk[u] < e;
        }
        if (e >= 0) place(e, s0 + rank, pos_q, type, box, perm, pos_q_sorted, type_sorted);
    }
}

// ---------------------------------------------------------------- fused MD-step passes

// One velocity-Verlet half step per atom and its cell: v += dt/2 a (when kick), x <-
// wrap(x + dt v), the float copy (x, y, z, q), the cell index and the histogram; the
// work of k_kick, k_drift_wrap and k_cell_index in one pass.  BATCHED: each atom's box
// from its system, cells numbered over the batch.
template <bool SMEM, bool BATCHED>
__global__ void __launch_bounds__(kStepThreads)
k_kick_drift_index(double *__restrict__ pos, double *__restrict__ vel, const void *__restrict__ forces,
                   int mode, const float *__restrict__ inv_mass, const float *__restrict__ q, int n,
                   BoxF box_in, BatchArgs b, double dt, double half_dt, int kick,
                   float4 *__restrict__ pos_q_out, int *__restrict__ cell_id,
                   int *__restrict__ cell_cnt, uint32_t *status)
{
    extern __shared__ int s_hist[];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int ncell = BATCHED ? b.ncell : box_in.ncell;
    if (SMEM) {
        for (int t = threadIdx.x; t < ncell; t += blockDim.x) s_hist[t] = 0;
        __syncthreads();
    }
    int c = -1;
    if (i < n) {
        const SysDesc *d = BATCHED ? &b.sys[b.atom_sys[i]] : nullptr;
        const BoxF &box = BATCHED ? d->box : box_in;
        double v[3] = {vel[3 * i], vel[3 * i + 1], vel[3 * i + 2]};
        if (kick) {
            double f[3];
            load_force(forces, mode, i, f);
            const double im = (double)inv_mass[i];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                v[k] = kick_velocity(v[k], f[k], im, half_dt);
                vel[3 * i + k] = v[k];
            }
        }
        double x[3];
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double w = drift_coord(pos[3 * i + k], v[k], dt);
            if (isfinite(w)) {
                w = wrap_coord(w, box.L[k]);
            } else {
                ok = false;
            }
            x[k] = w;
            pos[3 * i + k] = w;
        }
        if (!ok) set_status(status, MD_STATUS_NONFINITE);
        const float4 p = make_float4((float)x[0], (float)x[1], (float)x[2], q[i]);
        pos_q_out[i] = p;
        c = (BATCHED ? d->cell_offset : 0) + cell_of(p, box, status);
        cell_id[i] = c;
    }
    if (SMEM) {
        // one shared atomic per distinct cell of the warp (consecutive atoms often share
        // a cell)
        const unsigned act = __ballot_sync(0xffffffffu, c >= 0);
        const unsigned grp = __match_any_sync(0xffffffffu, c) & act;
        if (c >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&s_hist[c], __popc(grp));
        __syncthreads();
        for (int t = threadIdx.x; t < ncell; t += blockDim.x)
            if (s_hist[t]) atomicAdd(&cell_cnt[t], s_hist[t]);
    } else {
        const unsigned act = __ballot_sync(0xffffffffu, c >= 0);
        const unsigned grp = __match_any_sync(0xffffffffu, c) & act;
        if (c >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&cell_cnt[c], __popc(grp));
    }
}

constexpr int kClusterSortMax = 1024;  // cells with more members keep ascending input order

// One block per cell: the members straight into the force kernel's cluster order --
// columns of an S x S grid over the cell's x-y face, z along each column (alternating),
// ties by input index -- with the outputs of the cell build in that order (perm maps a
// slot to its input index).  This is a valid cell list (each cell contiguous); only the
// order within a cell differs from k_cell_sort's ascending input order.
template <bool BATCHED>
__global__ void __launch_bounds__(kSortThreads)
k_sort_cluster(const int *__restrict__ cell_start, const int *__restrict__ perm_tmp,
               const float4 *__restrict__ pos_q, const int32_t *__restrict__ type, BoxF box_in,
               BatchArgs b, int32_t *__restrict__ perm, float4 *__restrict__ pos_q_sorted,
               int32_t *__restrict__ type_sorted)
{
    __shared__ unsigned long long s_key[kClusterSortMax];
    const int cg = blockIdx.x;
    const BoxF &box = BATCHED ? b.sys[b.cell_sys[cg]].box : box_in;
    const int c = BATCHED ? cg - b.sys[b.cell_sys[cg]].cell_offset : cg;
    const int s0 = cell_start[cg];
    const int m = cell_start[cg + 1] - s0;
    if (m == 0) return;
    if (m > kClusterSortMax) {
        // ascending input index, as k_cell_sort
        int *chunk = reinterpret_cast<int *>(s_key);
        constexpr int kChunk = 2 * kClusterSortMax;
        for (int base = 0; base < m; base += kSortThreads) {
            const int t = base + threadIdx.x;
            const int e = t < m ? perm_tmp[s0 + t] : -1;
            int rank = 0;
            for (int c0 = 0; c0 < m; c0 += kChunk) {
                const int len = min(kChunk, m - c0);
                __syncthreads();
                for (int u = threadIdx.x; u < len; u += kSortThreads) chunk[u] = perm_tmp[s0 + c0 + u];
                __syncthreads();
                for (int u = 0; u < len; ++u) rank += chunk[u] < e;
            }
            if (e >= 0) place(e, s0 + rank, pos_q, type, box, perm, pos_q_sorted, type_sorted);
        }
        return;
    }
    const int nx = box.dims[0], ny = box.dims[1];
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    const int S = max(1, min(8, (int)(sqrtf((float)m * (1.0f / 20.0f)) + 0.5f)));
    for (int t = threadIdx.x; t < m; t += kSortThreads) {
        const int e = perm_tmp[s0 + t];
        const float4 p = pos_q[e];
        const double ux = wrap_coord((double)p.x, box.L[0]) * box.inv_edge[0] - cx;
        const double uy = wrap_coord((double)p.y, box.L[1]) * box.inv_edge[1] - cy;
        double uz = wrap_coord((double)p.z, box.L[2]) * box.inv_edge[2] - cz;
        const int kx = min(S - 1, max(0, (int)(ux * S))), ky = min(S - 1, max(0, (int)(uy * S)));
        const int col = ky * S + ((ky & 1) ? S - 1 - kx : kx);  // boustrophedon
        uz = fmin(fmax(uz, 0.0), 1.0);
        if (col & 1) uz = 1.0 - uz;
        const unsigned long long zq = (unsigned long long)(uz * 16777215.0);  // 24 bits
        // finite coordinates only matter for the order; e keeps the keys distinct
        s_key[t] = ((unsigned long long)col << 54) | (zq << 30) | (unsigned long long)e;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m; t += kSortThreads) {
        const unsigned long long key = s_key[t];
        int rank = 0;
        for (int u = 0; u < m; ++u) rank += s_key[u] < key;
        place((int)(key & ((1ull << 30) - 1)), s0 + rank, pos_q, type, box, perm, pos_q_sorted, type_sorted);
    }
}

}  // namespace

cudaError_t launch_build_cells(const float4 *pos_q, const int32_t *type, int n, const BoxF &box,
                               int32_t *cell_start, int32_t *perm, float4 *pos_q_sorted,
                               int32_t *type_sorted, const WsLayout &ws, char *wsp,
                               uint32_t *status, cudaStream_t stream)
{
    int *cell_id = reinterpret_cast<int *>(wsp + ws.cell_id);
    int *cnt = reinterpret_cast<int *>(wsp + ws.cell_cnt);
    int *perm_tmp = reinterpret_cast<int *>(wsp + ws.perm_tmp);
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)box.ncell, stream);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        int g = (n + kIndexThreads - 1) / kIndexThreads;
        if (box.ncell <= kSmemCells)
            k_cell_index<true><<<g, kIndexThreads, sizeof(int) * box.ncell, stream>>>(pos_q, n, box, cell_id, cnt, status);
        else
            k_cell_index<false><<<g, kIndexThreads, 0, stream>>>(pos_q, n, box, cell_id, cnt, status);
    }
    k_scan_cells<<<1, kScanThreads, 0, stream>>>(cnt, box.ncell, cell_start);
    if (n > 0) {
        int g = (n + kIndexThreads - 1) / kIndexThreads;
        k_scatter<<<g, kIndexThreads, 0, stream>>>(cell_id, n, cnt, perm_tmp);
        k_cell_sort<<<box.ncell, kSortThreads, 0, stream>>>(cell_start, perm_tmp, pos_q, type, box, perm,
                                                             pos_q_sorted, type_sorted);
    }
    return cudaGetLastError();
}

// The cell build of one velocity-Verlet step, fused: half kick (when kick), drift,
// wrap, float copy, cell index and histogram in one pass, then the scan, the scatter and
// the members of each cell straight into cluster order.  The outputs are a valid cell
// list whose within-cell order is the force kernel's cluster order.  BATCHED uses `b`
// (box_in is then unused).
cudaError_t launch_kick_drift_build(double *pos, double *vel, const void *forces, int mode,
                                    const float *inv_mass, const float *q, const int32_t *type, int n,
                                    const BoxF &box_in, const BatchArgs *b, double dt, double half_dt,
                                    bool kick, float4 *pos_q, int32_t *cell_start, int32_t *perm,
                                    float4 *pos_q_sorted, int32_t *type_sorted, const WsLayout &ws,
                                    char *wsp, uint32_t *status, cudaStream_t stream)
{
    int *cell_id = reinterpret_cast<int *>(wsp + ws.cell_id);
    int *cnt = reinterpret_cast<int *>(wsp + ws.cell_cnt);
    int *perm_tmp = reinterpret_cast<int *>(wsp + ws.perm_tmp);
    const int ncell = b ? b->ncell : box_in.ncell;
    const BatchArgs nob = {};
    const BatchArgs &bb = b ? *b : nob;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)ncell, stream);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        const int g = (n + kStepThreads - 1) / kStepThreads;
        const size_t sm = ncell <= kStepSmemCells ? sizeof(int) * (size_t)ncell : 0;
        const int k = kick ? 1 : 0;
        if (b) {
            if (sm) k_kick_drift_index<true, true><<<g, kStepThreads, sm, stream>>>(pos, vel, forces, mode, inv_mass, q, n, box_in, bb, dt, half_dt, k, pos_q, cell_id, cnt, status);
            else k_kick_drift_index<false, true><<<g, kStepThreads, 0, stream>>>(pos, vel, forces, mode, inv_mass, q, n, box_in, bb, dt, half_dt, k, pos_q, cell_id, cnt, status);
        } else {
            if (sm) k_kick_drift_index<true, false><<<g, kStepThreads, sm, stream>>>(pos, vel, forces, mode, inv_mass, q, n, box_in, bb, dt, half_dt, k, pos_q, cell_id, cnt, status);
            else k_kick_drift_index<false, false><<<g, kStepThreads, 0, stream>>>(pos, vel, forces, mode, inv_mass, q, n, box_in, bb, dt, half_dt, k, pos_q, cell_id, cnt, status);
        }
    }
    k_scan_cells<<<1, kScanThreads, 0, stream>>>(cnt, ncell, cell_start);
    if (n > 0) {
        const int g = (n + kIndexThreads - 1) / kIndexThreads;
        k_scatter<<<g, kIndexThreads, 0, stream>>>(cell_id, n, cnt, perm_tmp);
        if (b)
            k_sort_cluster<true><<<ncell, kSortThreads, 0, stream>>>(cell_start, perm_tmp, pos_q, type, box_in, bb, perm, pos_q_sorted, type_sorted);
        else
            k_sort_cluster<false><<<ncell, kSortThreads, 0, stream>>>(cell_start, perm_tmp, pos_q, type, box_in, bb, perm, pos_q_sorted, type_sorted);
    }
    return cudaGetLastError();
}

}  // namespace mdnb
