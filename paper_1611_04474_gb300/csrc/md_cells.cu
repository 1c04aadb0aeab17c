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
//
// The MD step fuses this with its integration (k_kick_drift_index: half kick, drift,
// wrap, cell index, count and a slot in a per-cell bin) and builds each cell straight
// in the force kernel's cluster order (k_sort_cluster), without the scan and the
// scatter when the bins hold every cell.
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
             int *__restrict__ cell_cnt, uint32_t *status, const int *__restrict__ run_flag)
{
    extern __shared__ int s_hist[];
    if (run_flag && !*run_flag) return;  // Verlet step without a rebuild
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
k_scan_cells(int *__restrict__ cnt_cursor, int ncell, int *__restrict__ cell_start,
             const int *__restrict__ run_flag)
{
    __shared__ int sums[kScanThreads];
    if (run_flag && !*run_flag) return;
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
k_scatter(const int *__restrict__ cell_id, int n, int *__restrict__ cursor, int *__restrict__ perm_tmp,
          const int *__restrict__ run_flag)
{
    if (run_flag && !*run_flag) return;
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

// Exclusive scan of ncell <= kStepSmemCells counts by one block of kStepThreads: the
// counts are staged in `s` (shared, ncell entries), cell_start[0..ncell] and the scatter
// cursors (= cell_start[c], in place of the counts) are written.
__device__ __forceinline__ void block_scan_cells(int *__restrict__ cnt_cursor, int ncell,
                                                 int *__restrict__ cell_start, int *s)
{
    __shared__ int warp_sum[kStepThreads / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int c = t; c < ncell; c += kStepThreads) s[c] = __ldcg(cnt_cursor + c);
    __syncthreads();
    const int per = (ncell + kStepThreads - 1) / kStepThreads;
    const int lo = min(t * per, ncell), hi = min(lo + per, ncell);
    int own = 0;
    for (int c = lo; c < hi; ++c) own += s[c];
    int incl = own;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    int before = 0;
#pragma unroll
    for (int w = 0; w < kStepThreads / 32; ++w) before += w < warp ? warp_sum[w] : 0;
    int run = before + incl - own;
    for (int c = lo; c < hi; ++c) {
        const int k = s[c];
        cell_start[c] = run;
        cnt_cursor[c] = run;
        run += k;
    }
    if (t == kStepThreads - 1) cell_start[ncell] = before + incl;
}

// One velocity-Verlet half step per atom and its cell: v += dt/2 a (when kick), x <-
// wrap(x + dt v), the float copy (x, y, z, q), the cell index and the histogram; the
// work of a kick, a drift with wrap and k_cell_index in one pass.  BATCHED: each atom's box
// from its system, cells numbered over the batch.  It also zeroes the force kernels'
// cluster-order accumulators (`accum`, MD_ACCUM_F32 float4[n] or MD_ACCUM_FIXED64
// u64[3][n]; null for none) and the persistent launches' item counters (`work`, may be
// null).  SMEM (ncell <= kStepSmemCells) without bins: the last block to finish also
// scans the histogram into cell_start and the scatter cursors; cell_cnt[ncell] counts
// finished blocks and must be zero at launch.  bin_cap > 0: each atom also takes a slot of its
// cell's bin (bins[c][0..bin_cap), by arrival; the count atomics hand out the slots),
// which replaces the scatter pass; members past bin_cap are not binned.
template <bool SMEM, bool BATCHED>
__global__ void __launch_bounds__(kStepThreads)
k_kick_drift_index(double *__restrict__ pos, double *__restrict__ vel, const void *__restrict__ forces,
                   int mode, const float *__restrict__ inv_mass, const float *__restrict__ q, int n,
                   BoxF box_in, BatchArgs b, double dt, double half_dt, int kick,
                   float4 *__restrict__ pos_q_out, int *__restrict__ cell_id,
                   int *__restrict__ cell_cnt, int *__restrict__ cell_start, void *__restrict__ accum,
                   int *__restrict__ work, int *__restrict__ bins, int bin_cap, uint32_t *status)
{
    extern __shared__ int s_hist[];
    pdl_trigger();  // the cell sort may be scheduled now; it waits for this pass
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int ncell = BATCHED ? b.ncell : box_in.ncell;
    if (SMEM) {
        for (int t = threadIdx.x; t < ncell; t += blockDim.x) s_hist[t] = 0;
        __syncthreads();
    }
    if (work && i < 2) work[i] = 0;
    int c = -1;
    if (i < n) {
        if (accum) {
            if (mode == MD_ACCUM_F32) {
                reinterpret_cast<float4 *>(accum)[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            } else {
                unsigned long long *A = reinterpret_cast<unsigned long long *>(accum);
                A[i] = 0ull;
                A[(size_t)n + i] = 0ull;
                A[2 * (size_t)n + i] = 0ull;
            }
        }
        const SysDesc *d = BATCHED ? &b.sys[b.atom_sys[i]] : nullptr;
        const BoxF &box = BATCHED ? d->box : box_in;
        double v[3] = {vel[3 * i], vel[3 * i + 1], vel[3 * i + 2]};
        if (kick) {
            double f[3];
            load_force(forces, mode, i, f);
            const double c = kick_factor((double)inv_mass[i], half_dt);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                v[k] = kick_velocity(v[k], f[k], c);
                vel[3 * i + k] = v[k];
            }
        }
        double x[3];
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double w = drift_coord(pos[3 * i + k], v[k], dt);
            if (!in_box_f64(w, box.L[k])) {
                if (isfinite(w))
                    w = wrap_coord(w, box.L[k]);
                else
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
    const int lane = threadIdx.x & 31;
    const unsigned act = __ballot_sync(0xffffffffu, c >= 0);
    const unsigned grp = __match_any_sync(0xffffffffu, c) & act;
    const int leader = __ffs(grp) - 1;
    const int below = __popc(grp & ((1u << lane) - 1u));  // members of the group before this lane
    if (SMEM) {
        // one shared atomic per distinct cell of the warp (consecutive atoms often share
        // a cell), then one global atomic per cell of the block
        int wb = 0;
        if (c >= 0 && lane == leader) wb = atomicAdd(&s_hist[c], __popc(grp));
        wb = __shfl_sync(0xffffffffu, wb, leader < 0 ? 0 : leader);
        __syncthreads();
        for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
            const int v = s_hist[t];
            if (v) {
                const int base = atomicAdd(&cell_cnt[t], v);
                if (bin_cap) s_hist[t] = base;  // the block's first slot in cell t
            }
        }
        if (bin_cap) {
            __syncthreads();
            if (c >= 0) {
                const int off = s_hist[c] + wb + below;
                if (off < bin_cap) bins[(size_t)c * bin_cap + off] = i;
            }
        }
        // without bins the last block to finish scans the counts for the scatter (each
        // block's adds are made visible before it is counted); with bins the cell sort
        // forms each cell's start itself
        if (!bin_cap) {
            __shared__ int s_last;
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) s_last = atomicAdd(&cell_cnt[ncell], 1) == (int)gridDim.x - 1;
            __syncthreads();
            if (s_last) {
                __threadfence();
                block_scan_cells(cell_cnt, ncell, cell_start, s_hist);
            }
        }
    } else {
        int base = 0;
        if (c >= 0 && lane == leader) base = atomicAdd(&cell_cnt[c], __popc(grp));
        base = __shfl_sync(0xffffffffu, base, leader < 0 ? 0 : leader);
        if (bin_cap && c >= 0) {
            const int off = base + below;
            if (off < bin_cap) bins[(size_t)c * bin_cap + off] = i;
        }
    }
}

constexpr int kClusterSortMax = 1024;  // cells with more members keep ascending input order
constexpr int kClusterCols = 64;       // at most 8 x 8 columns per cell

// One block per cell: the members straight into the force kernel's cluster order --
// columns of an S x S grid over the cell's x-y face, z along each column (alternating),
// ties by input index -- with the outputs of the cell build in that order (perm maps a
// slot to its input index).  This is a valid cell list (each cell contiguous); only the
// order within a cell differs from k_cell_sort's ascending input order.  The members
// are counted per column and each is ranked only against its own column's keys.  The
// order needs no particular rounding, only the same one every run, so the keys are
// formed in FP32.  The members come from the cell's bin (bin_cap > 0) or from the
// scatter (perm_tmp from cell_start); a cell whose members overflowed its bin gathers
// them, in ascending input order, from the cell ids of all n atoms.  counts (non-null,
// with bins): cell_start is formed here from the per-cell counts of all ncell cells.
template <bool BATCHED>
__global__ void __launch_bounds__(kSortThreads)
k_sort_cluster(int *__restrict__ cell_start, const int *__restrict__ perm_tmp,
               const int *__restrict__ bins, int bin_cap, const int *__restrict__ cell_id, int n,
               const int *__restrict__ counts, int ncell,
               const float4 *__restrict__ pos_q, const int32_t *__restrict__ type, BoxF box_in,
               BatchArgs b, int32_t *__restrict__ perm, float4 *__restrict__ pos_q_sorted,
               int32_t *__restrict__ type_sorted, const int *__restrict__ run_flag,
               float4 *__restrict__ x_ref, float4 *__restrict__ clu_box)
{
    // keys by arrival, then grouped by column; after the ranking, the cell's positions in
    // cluster order (for the cluster boxes)
    __shared__ __align__(16) unsigned long long s_kb[2 * kClusterSortMax];
    unsigned long long *s_key = s_kb, *s_bkt = s_kb + kClusterSortMax;
    __shared__ int s_col[kClusterCols + 1];                // counts, then column starts
    __shared__ int s_fill[kClusterCols];
    __shared__ int s_wcnt[kSortThreads / 32];
    __shared__ float4 s_pos[kClusterSortMax];  // wrapped positions + charges, by arrival
    __shared__ int s_typ[kClusterSortMax];     // types, by arrival
    pdl_wait();
    pdl_trigger();
    if (run_flag && !*run_flag) return;  // Verlet step without a rebuild
    const int cg = blockIdx.x;
    const BoxF &box = BATCHED ? b.sys[b.cell_sys[cg]].box : box_in;
    const int c = BATCHED ? cg - b.sys[b.cell_sys[cg]].cell_offset : cg;
    // Verlet step: each member's position at this rebuild (input order), from what
    // place() or the staged copy writes
    auto put = [&](int e, int slot) {
        place(e, slot, pos_q, type, box, perm, pos_q_sorted, type_sorted);
        if (x_ref) x_ref[e] = pos_q_sorted[slot];
    };
    int s0, m;
    if (counts) {
        // this cell's start from the counts of the cells before it (a block sum), and
        // cell_start written here
        m = __ldcg(counts + cg);
        int part = 0;
        for (int t = threadIdx.x; t < cg; t += kSortThreads) part += __ldcg(counts + t);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((threadIdx.x & 31) == 0) s_wcnt[threadIdx.x >> 5] = part;
        __syncthreads();
        s0 = 0;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) s0 += s_wcnt[w];
        __syncthreads();
        if (threadIdx.x == 0) {
            cell_start[cg] = s0;
            if (cg == ncell - 1) cell_start[ncell] = s0 + m;
        }
    } else {
        s0 = cell_start[cg];
        m = cell_start[cg + 1] - s0;
    }
    if (m == 0) return;
    // cluster boxes (clu_box): after the cell's atoms are written, from what was written
    auto boxes = [&]() {
        if (!clu_box) return;
        __syncthreads();
        write_cluster_boxes<kSortThreads>(pos_q_sorted + s0, s0, m, clu_box, n);
    };
    const int *mem = bin_cap ? bins + (size_t)cg * bin_cap : perm_tmp + s0;
    if (bin_cap && m > bin_cap) {
        // ordered gather: members in ascending input order, placed directly when the
        // cell is too large for the cluster order, else listed for it (in s_bkt)
        int *list = reinterpret_cast<int *>(s_bkt);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int found = 0;
        for (int base = 0; base < n; base += kSortThreads) {
            const int j = base + threadIdx.x;
            const bool mine = j < n && cell_id[j] == cg;
            const unsigned bal = __ballot_sync(0xffffffffu, mine);
            if (lane == 0) s_wcnt[warp] = __popc(bal);
            __syncthreads();
            int before = found, total = found;
#pragma unroll
            for (int w = 0; w < kSortThreads / 32; ++w) {
                before += w < warp ? s_wcnt[w] : 0;
                total += s_wcnt[w];
            }
            const int pos = before + __popc(bal & ((1u << lane) - 1u));
            if (mine && pos < m) {
                if (m > kClusterSortMax)
                    put(j, s0 + pos);
                else
                    list[pos] = j;
            }
            found = total;
            __syncthreads();
        }
        if (m > kClusterSortMax) {
            boxes();
            return;
        }
        mem = list;
    } else if (m > kClusterSortMax) {
        // ascending input index, as k_cell_sort
        int *chunk = reinterpret_cast<int *>(s_key);
        constexpr int kChunk = 2 * kClusterSortMax;
        for (int base = 0; base < m; base += kSortThreads) {
            const int t = base + threadIdx.x;
            const int e = t < m ? mem[t] : -1;
            int rank = 0;
            for (int c0 = 0; c0 < m; c0 += kChunk) {
                const int len = min(kChunk, m - c0);
                __syncthreads();
                for (int u = threadIdx.x; u < len; u += kSortThreads) chunk[u] = mem[c0 + u];
                __syncthreads();
                for (int u = 0; u < len; ++u) rank += chunk[u] < e;
            }
            if (e >= 0) put(e, s0 + rank);
        }
        boxes();
        return;
    }
    const int nx = box.dims[0], ny = box.dims[1];
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    const int S = max(1, min(8, (int)(sqrtf((float)m * (1.0f / 20.0f)) + 0.5f)));
    const int ncol = S * S;
    for (int t = threadIdx.x; t < ncol; t += kSortThreads) {
        s_col[t] = 0;
        s_fill[t] = 0;
    }
    __syncthreads();
    const float fS = (float)S;
    for (int t = threadIdx.x; t < m; t += kSortThreads) {
        const int e = mem[t];
        const float4 p = wrap_pos_f(pos_q[e], box);
        s_pos[t] = p;
        s_typ[t] = type[e];
        // position in cell units, clamped onto the cell's faces
        const float ux = __fsub_rn(__fmul_rn(p.x, box.inv_edge_f[0]), (float)cx);
        const float uy = __fsub_rn(__fmul_rn(p.y, box.inv_edge_f[1]), (float)cy);
        float uz = __fsub_rn(__fmul_rn(p.z, box.inv_edge_f[2]), (float)cz);
        const int kx = min(S - 1, max(0, (int)__fmul_rn(ux, fS)));
        const int ky = min(S - 1, max(0, (int)__fmul_rn(uy, fS)));
        const int col = ky * S + ((ky & 1) ? S - 1 - kx : kx);  // boustrophedon
        uz = fminf(fmaxf(uz, 0.0f), 1.0f);
        if (col & 1) uz = __fsub_rn(1.0f, uz);
        const unsigned long long zq = (unsigned long long)(unsigned)__fmul_rn(uz, 16777215.0f);  // 24 bits
        // finite coordinates only matter for the order; e keeps the keys distinct
        s_key[t] = ((unsigned long long)col << 54) | (zq << 30) | (unsigned long long)e;
        atomicAdd(&s_col[col], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < ncol; ++k) {
            const int v = s_col[k];
            s_col[k] = run;
            run += v;
        }
        s_col[ncol] = run;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m; t += kSortThreads) {
        const unsigned long long key = s_key[t];
        const int col = (int)(key >> 54);
        s_bkt[s_col[col] + atomicAdd(&s_fill[col], 1)] = key;
    }
    __syncthreads();
    constexpr int kPer = kClusterSortMax / kSortThreads;  // members per thread at most
    int rk[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int t = threadIdx.x + i * kSortThreads;
        rk[i] = -1;
        if (t < m) {
            const unsigned long long key = s_key[t];
            const int col = (int)(key >> 54);
            const int b0 = s_col[col], b1 = s_col[col + 1];
            int rank = 0;
            for (int u = b0; u < b1; ++u) rank += s_bkt[u] < key;
            // what place() writes, from the copies staged above
            const int slot = s0 + b0 + rank;
            const int e = (int)(key & ((1ull << 30) - 1));
            perm[slot] = e;
            pos_q_sorted[slot] = s_pos[t];
            type_sorted[slot] = s_typ[t];
            if (x_ref) x_ref[e] = s_pos[t];
            rk[i] = b0 + rank;
        }
    }
    if (clu_box) {
        // the cluster boxes from the positions placed in shared memory in cluster order
        float4 *s_ord = reinterpret_cast<float4 *>(s_kb);
        __syncthreads();  // every rank formed: the keys are no longer read
#pragma unroll
        for (int i = 0; i < kPer; ++i)
            if (rk[i] >= 0) s_ord[rk[i]] = s_pos[threadIdx.x + i * kSortThreads];
        __syncthreads();
        write_cluster_boxes<kSortThreads>(s_ord, s0, m, clu_box, n);
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
            k_cell_index<true><<<g, kIndexThreads, sizeof(int) * box.ncell, stream>>>(pos_q, n, box, cell_id, cnt, status, nullptr);
        else
            k_cell_index<false><<<g, kIndexThreads, 0, stream>>>(pos_q, n, box, cell_id, cnt, status, nullptr);
    }
    k_scan_cells<<<1, kScanThreads, 0, stream>>>(cnt, box.ncell, cell_start, nullptr);
    if (n > 0) {
        int g = (n + kIndexThreads - 1) / kIndexThreads;
        k_scatter<<<g, kIndexThreads, 0, stream>>>(cell_id, n, cnt, perm_tmp, nullptr);
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
    void *accum = mode == MD_ACCUM_F64 ? nullptr : static_cast<void *>(wsp + ws.accum);
    int *work = reinterpret_cast<int *>(wsp + ws.work);
    int *bins = reinterpret_cast<int *>(wsp + ws.bins);
    const int cap = ws.bin_cap;
    const int ncell = b ? b->ncell : box_in.ncell;
    const BatchArgs nob = {};
    const BatchArgs &bb = b ? *b : nob;
    // the counts and the finished-block counter
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)ncell + 1), stream);
    if (e != cudaSuccess) return e;
    const size_t sm = ncell <= kStepSmemCells ? sizeof(int) * (size_t)ncell : 0;
    if (n > 0) {
        const int g = (n + kStepThreads - 1) / kStepThreads;
        const int k = kick ? 1 : 0;
        if (b) {
            if (sm) k_kick_drift_index<true, true><<<g, kStepThreads, sm, stream>>>(pos, vel, forces, mode, inv_mass, q, n, box_in, bb, dt, half_dt, k, pos_q, cell_id, cnt, cell_start, accum, work, bins, cap, status);
            else k_kick_drift_index<false, true><<<g, kStepThreads, 0, stream>>>(pos, vel, forces, mode, inv_mass, q, n, box_in, bb, dt, half_dt, k, pos_q, cell_id, cnt, cell_start, accum, work, bins, cap, status);
        } else {
            if (sm) k_kick_drift_index<true, false><<<g, kStepThreads, sm, stream>>>(pos, vel, forces, mode, inv_mass, q, n, box_in, bb, dt, half_dt, k, pos_q, cell_id, cnt, cell_start, accum, work, bins, cap, status);
            else k_kick_drift_index<false, false><<<g, kStepThreads, 0, stream>>>(pos, vel, forces, mode, inv_mass, q, n, box_in, bb, dt, half_dt, k, pos_q, cell_id, cnt, cell_start, accum, work, bins, cap, status);
        }
    }
    // the shared-histogram form scans in its last block (without bins) or in the cell
    // sort (with bins)
    const bool sort_scans = n > 0 && sm && cap;
    if (n == 0 || !sm) k_scan_cells<<<1, kScanThreads, 0, stream>>>(cnt, ncell, cell_start, nullptr);
    if (n > 0) {
        // with bins the members are already grouped by cell
        if (!cap) {
            const int g = (n + kIndexThreads - 1) / kIndexThreads;
            k_scatter<<<g, kIndexThreads, 0, stream>>>(cell_id, n, cnt, perm_tmp, nullptr);
        }
        // after the scatter, or straight after the build pass (programmatic launch)
        if (b)
            e = launch_pdl(k_sort_cluster<true>, dim3(ncell), dim3(kSortThreads), 0, stream, cell_start, perm_tmp, bins, cap, (const int *)cell_id, n, sort_scans ? (const int *)cnt : nullptr, ncell, (const float4 *)pos_q, type, box_in, bb, perm, pos_q_sorted, type_sorted, (const int *)nullptr, (float4 *)nullptr, (float4 *)nullptr);
        else
            e = launch_pdl(k_sort_cluster<false>, dim3(ncell), dim3(kSortThreads), 0, stream, cell_start, perm_tmp, bins, cap, (const int *)cell_id, n, sort_scans ? (const int *)cnt : nullptr, ncell, (const float4 *)pos_q, type, box_in, bb, perm, pos_q_sorted, type_sorted, (const int *)nullptr, (float4 *)nullptr, reinterpret_cast<float4 *>(wsp + ws.clu_box));
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// The cell rebuild of a Verlet step (md_step_verlet): the counting sort of the input-order
// float positions into the cells of the Verlet grid, each cell's members straight into
// cluster order, and x_ref[i] = the position each atom has at this rebuild.  Every kernel
// reads *run_flag first and returns at once when it is 0 (no rebuild this step), so the
// launches can be enqueued every step without a host decision.
cudaError_t launch_verlet_rebuild(const float4 *pos_q, const int32_t *type, int n, const BoxF &box,
                                  int32_t *cell_start, int32_t *perm, float4 *pos_q_sorted,
                                  int32_t *type_sorted, float4 *x_ref, const int *run_flag,
                                  const WsLayout &ws, char *wsp, uint32_t *status,
                                  cudaStream_t stream)
{
    int *cell_id = reinterpret_cast<int *>(wsp + ws.cell_id);
    int *cnt = reinterpret_cast<int *>(wsp + ws.cell_cnt);
    int *perm_tmp = reinterpret_cast<int *>(wsp + ws.perm_tmp);
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)box.ncell + 1), stream);
    if (e != cudaSuccess || n <= 0) return e;
    const int g = (n + kIndexThreads - 1) / kIndexThreads;
    if (box.ncell <= kSmemCells)
        k_cell_index<true><<<g, kIndexThreads, sizeof(int) * box.ncell, stream>>>(pos_q, n, box, cell_id, cnt, status, run_flag);
    else
        k_cell_index<false><<<g, kIndexThreads, 0, stream>>>(pos_q, n, box, cell_id, cnt, status, run_flag);
    k_scan_cells<<<1, kScanThreads, 0, stream>>>(cnt, box.ncell, cell_start, run_flag);
    k_scatter<<<g, kIndexThreads, 0, stream>>>(cell_id, n, cnt, perm_tmp, run_flag);
    const BatchArgs nob = {};
    k_sort_cluster<false><<<box.ncell, kSortThreads, 0, stream>>>(
        cell_start, perm_tmp, (const int *)nullptr, 0, (const int *)cell_id, n, (const int *)nullptr,
        box.ncell, pos_q, type, box, nob, perm, pos_q_sorted, type_sorted, run_flag, x_ref,
        (float4 *)nullptr);
    return cudaGetLastError();
}

}  // namespace mdnb
