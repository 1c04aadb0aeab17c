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

constexpr int kIndexThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kSortThreads = 128;
constexpr int kSortChunk = 2048;  // members staged in shared memory at a time

__device__ __forceinline__ bool finite3(double x, double y, double z)
{
    return isfinite(x) && isfinite(y) && isfinite(z);
}

__global__ void __launch_bounds__(kIndexThreads)
k_cell_index(const float4 *__restrict__ pos_q, int n, BoxF box, int *__restrict__ cell_id,
             int *__restrict__ cell_cnt, uint32_t *status)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 p = pos_q[i];
    double x = p.x, y = p.y, z = p.z;
    int c = 0;
    if (finite3(x, y, z)) {
        int cx = cell_coord(wrap_coord(x, box.L[0]), box.dims[0], box.L[0]);
        int cy = cell_coord(wrap_coord(y, box.L[1]), box.dims[1], box.L[1]);
        int cz = cell_coord(wrap_coord(z, box.L[2]), box.dims[2], box.L[2]);
        c = cx + box.dims[0] * (cy + box.dims[1] * cz);
    } else {
        set_status(status, MD_STATUS_NONFINITE);
    }
    cell_id[i] = c;
    atomicAdd(&cell_cnt[c], 1);
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

__global__ void __launch_bounds__(kIndexThreads)
k_scatter(const int *__restrict__ cell_id, int n, int *__restrict__ cursor, int *__restrict__ perm_tmp)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int slot = atomicAdd(&cursor[cell_id[i]], 1);
    perm_tmp[slot] = i;
}

// One block per cell.  Members are distinct input indices, so the rank of a member
// among them (number of smaller members) is its slot in ascending input order.
__global__ void __launch_bounds__(kSortThreads)
k_cell_sort(const int *__restrict__ cell_start, const int *__restrict__ perm_tmp,
            const float4 *__restrict__ pos_q, const int32_t *__restrict__ type, BoxF box,
            int32_t *__restrict__ perm, float4 *__restrict__ pos_q_sorted,
            int32_t *__restrict__ type_sorted)
{
    __shared__ int chunk[kSortChunk];
    int c = blockIdx.x;
    int s0 = cell_start[c];
    int m = cell_start[c + 1] - s0;
    if (m == 0) return;
    // each thread owns members t, t + blockDim, ...; ranks accumulate chunk by chunk
    constexpr int kOwn = (kSortChunk + kSortThreads - 1) / kSortThreads;  // when m fits one chunk
    int own_val[kOwn];
    int own_rank[kOwn];
    int rounds = (m + kSortThreads - 1) / kSortThreads;
    // members beyond kOwn rounds are handled by re-reading perm_tmp (large cells only)
    for (int base = 0; base < rounds; base += kOwn) {
        int nr = min(kOwn, rounds - base);
        for (int r = 0; r < kOwn; ++r) {
            int t = (base + r) * kSortThreads + threadIdx.x;
            own_val[r] = (r < nr && t < m) ? perm_tmp[s0 + t] : -1;
            own_rank[r] = 0;
        }
        for (int c0 = 0; c0 < m; c0 += kSortChunk) {
            int len = min(kSortChunk, m - c0);
            __syncthreads();
            for (int u = threadIdx.x; u < len; u += kSortThreads) chunk[u] = perm_tmp[s0 + c0 + u];
            __syncthreads();
            for (int u = 0; u < len; ++u) {
                int v = chunk[u];
#pragma unroll
                for (int r = 0; r < kOwn; ++r) own_rank[r] += (v < own_val[r]);
            }
        }
        for (int r = 0; r < kOwn; ++r) {
            int e = own_val[r];
            if (e < 0) continue;
            int slot = s0 + own_rank[r];
            perm[slot] = e;
            float4 p = pos_q[e];
            double x = p.x, y = p.y, z = p.z;
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
        k_cell_index<<<g, kIndexThreads, 0, stream>>>(pos_q, n, box, cell_id, cnt, status);
    }
    k_scan_cells<<<1, kScanThreads, 0, stream>>>(cnt, box.ncell, cell_start);
    if (n > 0) {
        int g = (n + kIndexThreads - 1) / kIndexThreads;
        k_scatter<<<g, kIndexThreads, 0, stream>>>(cell_id, n, cnt, perm_tmp);
        k_cell_sort<<<box.ncell, kSortThreads, 0, stream>>>(cell_start, perm_tmp, pos_q, type, box,
                                                             perm, pos_q_sorted, type_sorted);
    }
    return cudaGetLastError();
}

}  // namespace mdnb
