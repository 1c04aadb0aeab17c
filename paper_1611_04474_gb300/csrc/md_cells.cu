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
constexpr int kSmemCells = 8192;     // per-block shared histogram up to this many cells
constexpr int kScanThreads = 1024;
constexpr int kSortThreads = 128;
constexpr int kSortChunk = 2048;  // members staged in shared memory at a time

__device__ __forceinline__ bool finite3(double x, double y, double z)
{
    return isfinite(x) && isfinite(y) && isfinite(z);
}

__device__ __forceinline__ int cell_of(const float4 &p, const BoxF &box, uint32_t *status)
{
    double x = p.x, y = p.y, z = p.z;
    if (!finite3(x, y, z)) {
        set_status(status, MD_STATUS_NONFINITE);
        return 0;
    }
    int cx = cell_coord(wrap_coord(x, box.L[0]), box.dims[0], box.inv_edge[0]);
    int cy = cell_coord(wrap_coord(y, box.L[1]), box.dims[1], box.inv_edge[1]);
    int cz = cell_coord(wrap_coord(z, box.L[2]), box.dims[2], box.inv_edge[2]);
    return cx + box.dims[0] * (cy + box.dims[1] * cz);
}

// Per-block histogram in shared memory (grids with up to kSmemCells cells), then one
// global add per touched cell; larger grids count with warp-aggregated global atomics.
// Batched: every atom's box comes from its system and cells are numbered globally.
template <bool SMEM, bool BATCHED>
__global__ void __launch_bounds__(kIndexThreads)
k_cell_index(const float4 *__restrict__ pos_q, int n, BoxF box, BatchArgs b,
             int *__restrict__ cell_id, int *__restrict__ cell_cnt, uint32_t *status)
{
    extern __shared__ int s_hist[];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int ncell = BATCHED ? b.ncell : box.ncell;
    if (SMEM) {
        for (int t = threadIdx.x; t < ncell; t += blockDim.x) s_hist[t] = 0;
        __syncthreads();
    }
    int c = -1;
    if (i < n) {
        if (BATCHED) {
            const SysDesc &d = b.sys[b.atom_sys[i]];
            c = d.cell_offset + cell_of(pos_q[i], d.box, status);
        } else {
            c = cell_of(pos_q[i], box, status);
        }
        cell_id[i] = c;
    }
    if (SMEM) {
        if (c >= 0) atomicAdd(&s_hist[c], 1);
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
__device__ __forceinline__ void place(int e, int slot, const float4 *__restrict__ pos_q,
                                      const int32_t *__restrict__ type, const BoxF &box,
                                      int32_t *__restrict__ perm, float4 *__restrict__ pos_q_sorted,
                                      int32_t *__restrict__ type_sorted)
{
    perm[slot] = e;
    const float4 p = pos_q[e];
    const double x = p.x, y = p.y, z = p.z;
    float4 o;
    if (finite3(x, y, z)) {
        o.x = (float)wrap_coord(x, box.L[0]);
        o.y = (float)wrap_coord(y, box.L[1]);
        o.z = (float)wrap_coord(z, box.L[2]);
    } else {
        o.x = o.y = o.z = 0.0f;
    }
    o.w = p.w;
    pos_q_sorted[slot] = o;
    type_sorted[slot] = type[e];
}

template <bool BATCHED>
__global__ void __launch_bounds__(kSortThreads)
k_cell_sort(const int *__restrict__ cell_start, const int *__restrict__ perm_tmp,
            const float4 *__restrict__ pos_q, const int32_t *__restrict__ type, BoxF box_in,
            BatchArgs b, int32_t *__restrict__ perm, float4 *__restrict__ pos_q_sorted,
            int32_t *__restrict__ type_sorted)
{
    __shared__ int chunk[kSortChunk];
    const int c = blockIdx.x;
    const BoxF &box = BATCHED ? b.sys[b.cell_sys[c]].box : box_in;
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
    BatchArgs nob = {};
    if (n > 0) {
        int g = (n + kIndexThreads - 1) / kIndexThreads;
        if (box.ncell <= kSmemCells)
            k_cell_index<true, false><<<g, kIndexThreads, sizeof(int) * box.ncell, stream>>>(pos_q, n, box, nob, cell_id, cnt, status);
        else
            k_cell_index<false, false><<<g, kIndexThreads, 0, stream>>>(pos_q, n, box, nob, cell_id, cnt, status);
    }
    k_scan_cells<<<1, kScanThreads, 0, stream>>>(cnt, box.ncell, cell_start);
    if (n > 0) {
        int g = (n + kIndexThreads - 1) / kIndexThreads;
        k_scatter<<<g, kIndexThreads, 0, stream>>>(cell_id, n, cnt, perm_tmp);
        k_cell_sort<false><<<box.ncell, kSortThreads, 0, stream>>>(cell_start, perm_tmp, pos_q, type, box,
                                                                    nob, perm, pos_q_sorted, type_sorted);
    }
    return cudaGetLastError();
}

cudaError_t launch_build_cells_batched(const float4 *pos_q, const int32_t *type, const BatchArgs &b,
                                       int32_t *cell_start, int32_t *perm, float4 *pos_q_sorted,
                                       int32_t *type_sorted, const WsLayout &ws, char *wsp,
                                       uint32_t *status, cudaStream_t stream)
{
    int *cell_id = reinterpret_cast<int *>(wsp + ws.cell_id);
    int *cnt = reinterpret_cast<int *>(wsp + ws.cell_cnt);
    int *perm_tmp = reinterpret_cast<int *>(wsp + ws.perm_tmp);
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)b.ncell, stream);
    if (e != cudaSuccess) return e;
    BoxF nobox = {};
    const int n = b.n;
    if (n > 0) {
        int g = (n + kIndexThreads - 1) / kIndexThreads;
        if (b.ncell <= kSmemCells)
            k_cell_index<true, true><<<g, kIndexThreads, sizeof(int) * b.ncell, stream>>>(pos_q, n, nobox, b, cell_id, cnt, status);
        else
            k_cell_index<false, true><<<g, kIndexThreads, 0, stream>>>(pos_q, n, nobox, b, cell_id, cnt, status);
    }
    k_scan_cells<<<1, kScanThreads, 0, stream>>>(cnt, b.ncell, cell_start);
    if (n > 0) {
        int g = (n + kIndexThreads - 1) / kIndexThreads;
        k_scatter<<<g, kIndexThreads, 0, stream>>>(cell_id, n, cnt, perm_tmp);
        k_cell_sort<true><<<b.ncell, kSortThreads, 0, stream>>>(cell_start, perm_tmp, pos_q, type, nobox,
                                                                 b, perm, pos_q_sorted, type_sorted);
    }
    return cudaGetLastError();
}

}  // namespace mdnb
