// md_forces_cluster.cu -- cluster-pair force kernel (MD_ALGO_CLUSTER).
//
// The same half shell of cell pairs as MD_ALGO_HALF_SHELL (each unordered pair once,
// the reaction by Newton's third law), with the filter/force split of the paper's
// enhanced accelerator (Section V.B) placed one level higher: the candidates are
// filtered by whole groups of atoms and the force stage runs on every pair of a group
// pair that survives.
//
//   order:   each cell's atoms are reordered into spatially compact groups: columns
//            of an S x S grid over the cell's x-y face, each column sorted along z
//            (alternating direction), so that consecutive atoms are neighbours.  A
//            home cell is cut into i-clusters of 4 atoms, a neighbour cell into
//            j-clusters of 8.
//   filter:  one lane per j-cluster tests the gap between the bounding boxes of the
//            i-cluster and 32 j-clusters at once (rc'^2, conservative); a ballot
//            lists the j-clusters in range (about 39% of their 32 pairs are within
//            rc on the dense workloads, against 14% of the cell-pair candidates).
//   force:   a warp evaluates the 4 x 8 pairs of one cluster pair, one pair per lane
//            (lane = i + 4 j), with the exact test r^2 < rc^2 per pair.
//   reduce:  i-forces stay in registers for the whole i-cluster; the reaction on each
//            j atom is summed over its 4 lanes with two shuffles and added to a
//            warp-private shared array (no atomics inside a tile).
//
// The pair arithmetic is the library's (pair_r2, pair_f, the same staged coordinates
// and shifts as the half-shell kernel), so MD_ACCUM_FIXED64 results are the same bits
// as the other kernels'.  Boxes with an axis of 2 cells use the half-shell kernel.
#include <math.h>

#include "md_internal.cuh"
#include "md_pairgeom.cuh"

namespace mdnb {
namespace {

constexpr int kCI = 4;         // atoms per i-cluster (home cell)
constexpr int kCJ = 8;         // atoms per j-cluster (neighbour cell)
constexpr int kCW = 4;         // warps per CTA
constexpr int kCT = kCW * 32;  // threads per CTA
constexpr int kCTile = 256;    // atoms of a cell staged at once (multiple of kCJ)
constexpr int kSortMax = 1024; // cells with more atoms keep their sorted order
constexpr int kOrderThreads = 256;

static_assert(kCI * kCJ == 32, "one cluster pair per warp");
static_assert(kCTile % kCJ == 0 && kCTile % kCI == 0, "tiles hold whole clusters");

// Per cell: sort its atoms by (column, z along the column) and write the reordered
// copies.  corder[k] is the sorted-order slot of cluster-order slot k.
__global__ void __launch_bounds__(kOrderThreads)
k_cluster_order(const int32_t *__restrict__ cell_start, const float4 *__restrict__ pq,
                const int32_t *__restrict__ ty, BoxF box, float4 *__restrict__ cpq,
                int32_t *__restrict__ cty, int32_t *__restrict__ corder)
{
    __shared__ unsigned long long s_key[kSortMax];
    const int c = blockIdx.x;
    const int b = cell_start[c], m = cell_start[c + 1] - b;
    if (m <= 0) return;
    if (m > kSortMax) {
        for (int t = threadIdx.x; t < m; t += kOrderThreads) {
            corder[b + t] = b + t;
            cpq[b + t] = pq[b + t];
            cty[b + t] = ty[b + t];
        }
        return;
    }
    const int nx = box.dims[0], ny = box.dims[1];
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    // about 20 atoms per column
    const int S = max(1, min(8, (int)(sqrtf((float)m * (1.0f / 20.0f)) + 0.5f)));
    const float ex = (float)box.inv_edge[0], ey = (float)box.inv_edge[1], ez = (float)box.inv_edge[2];
    for (int t = threadIdx.x; t < m; t += kOrderThreads) {
        const float4 p = pq[b + t];
        const float ux = fminf(fmaxf(p.x * ex - (float)cx, 0.0f), 0.999999f);
        const float uy = fminf(fmaxf(p.y * ey - (float)cy, 0.0f), 0.999999f);
        float uz = fminf(fmaxf(p.z * ez - (float)cz, 0.0f), 1.0f);
        const int kx = (int)(ux * (float)S), ky = (int)(uy * (float)S);
        const int col = ky * S + ((ky & 1) ? S - 1 - kx : kx);  // boustrophedon
        if (col & 1) uz = 1.0f - uz;
        const unsigned zq = (unsigned)(uz * 1048575.0f);
        s_key[t] = ((unsigned long long)col << 44) | ((unsigned long long)zq << 20) |
                   (unsigned long long)t;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m; t += kOrderThreads) {
        const unsigned long long k = s_key[t];
        int rank = 0;
        for (int u = 0; u < m; ++u) rank += s_key[u] < k;
        corder[b + rank] = b + t;
        cpq[b + rank] = pq[b + t];
        cty[b + rank] = ty[b + t];
    }
}

struct CluArgs {
    const int32_t *cell_start;
    const float4 *pq;   // cluster order
    const int32_t *ty;  // cluster order
    BoxF box;
    const float2 *AB;
    int ntypes;
    float kc;
    float rc2;   // exact cutoff test
    float rc2m;  // cluster filter threshold (conservative)
    void *accum; // float4[n] (F32) or u64[3][n] (FIXED64), cluster order, zeroed
    int n;
    Partial *partials;
    uint32_t *status;
};

// Bounding boxes of the clusters of a staged tile (padding excluded).
template <int CS>
__device__ __forceinline__ void cluster_boxes(const float4 *p, int m, float (*box)[6])
{
    const int nclu = (m + CS - 1) / CS;
    for (int k = threadIdx.x; k < nclu; k += kCT) {
        float lo[3] = {kFar, kFar, kFar}, hi[3] = {-kFar, -kFar, -kFar};
        const int e = min(m, (k + 1) * CS);
        for (int t = k * CS; t < e; ++t) {
            const float4 q = p[t];
            lo[0] = fminf(lo[0], q.x); hi[0] = fmaxf(hi[0], q.x);
            lo[1] = fminf(lo[1], q.y); hi[1] = fmaxf(hi[1], q.y);
            lo[2] = fminf(lo[2], q.z); hi[2] = fmaxf(hi[2], q.z);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            box[k][d] = lo[d];
            box[k][d + 3] = hi[d];
        }
    }
}

template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(kCT, MODE == MD_ACCUM_FIXED64 ? 5 : 7)
k_cluster(CluArgs a)
{
    using Acc = typename AccT<MODE>::T;
    __shared__ __align__(16) float4 s_hp[kCTile];  // home tile (x, y, z shifted, q)
    __shared__ __align__(16) float4 s_np[kCTile];  // neighbour tile
    __shared__ int s_ht[kCTile], s_nt[kCTile];
    __shared__ float s_ib[kCTile / kCI][6];  // i-cluster boxes: lo xyz, hi xyz
    __shared__ float s_jb[kCTile / kCJ][6];  // j-cluster boxes
    __shared__ Acc s_hf[3][kCTile];          // forces on home atoms (whole cell pair)
    __shared__ Acc s_nf[kCW][3][kCTile];     // per-warp reactions on neighbour atoms (tile)
    extern __shared__ __align__(16) unsigned char s_dyn[];
    float2 *s_ab = reinterpret_cast<float2 *>(s_dyn);  // LJ table [ntypes * ntypes]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int il = lane & (kCI - 1), jl = lane / kCI;
    float e_lj = 0.f, e_c = 0.f, vir = 0.f;
    unsigned long long cnt = 0;
    Partial *mine = a.partials + (size_t)blockIdx.y * gridDim.x;

    PairGeom g;
    if (!cell_pair(a.box, blockIdx.x, blockIdx.y, g)) {
        block_partial<kCT>(0.0, 0.0, 0.0, 0ull, mine);
        return;
    }
    const int h_begin = a.cell_start[g.home], nh = a.cell_start[g.home + 1] - h_begin;
    const int n_begin = a.cell_start[g.nbr], nn = a.cell_start[g.nbr + 1] - n_begin;
    if (nh == 0 || nn == 0) {
        block_partial<kCT>(0.0, 0.0, 0.0, 0ull, mine);
        return;
    }
    const int T = a.ntypes;
    for (int t = threadIdx.x; t < T * T; t += kCT) s_ab[t] = a.AB[t];
    const float kc = a.kc, rc2 = a.rc2, rc2m = a.rc2m;

    for (int h0 = 0; h0 < nh; h0 += kCTile) {
        const int mh = min(kCTile, nh - h0);
        const int nic = (mh + kCI - 1) / kCI;
        __syncthreads();
        for (int t = threadIdx.x; t < nic * kCI; t += kCT) {
            float4 p;
            int ty = 0;
            if (t < mh) {
                p = a.pq[h_begin + h0 + t];
                p.x -= g.hs[0];
                p.y -= g.hs[1];
                p.z -= g.hs[2];
                ty = clamp_type(a.ty[h_begin + h0 + t], T, a.status);
            } else {
                p = make_float4(kFar, kFar, kFar, 0.f);
            }
            s_hp[t] = p;
            s_ht[t] = ty;
            s_hf[0][t] = s_hf[1][t] = s_hf[2][t] = Acc(0);
        }
        __syncthreads();
        cluster_boxes<kCI>(s_hp, mh, s_ib);
        for (int n0 = g.self ? h0 : 0; n0 < nn; n0 += kCTile) {
            const int mn = min(kCTile, nn - n0);
            const int njc = (mn + kCJ - 1) / kCJ;
            const bool diag = g.self && n0 == h0;
            __syncthreads();
            for (int t = threadIdx.x; t < njc * kCJ; t += kCT) {
                float4 p;
                int ty = 0;
                if (t >= mn) {
                    p = make_float4(-kFar, -kFar, -kFar, 0.f);
                } else if (diag) {
                    p = s_hp[t];  // the home tile holds the same atoms
                    ty = s_ht[t];
                } else {
                    p = a.pq[n_begin + n0 + t];
                    p.x -= g.ns[0];
                    p.y -= g.ns[1];
                    p.z -= g.ns[2];
                    ty = clamp_type(a.ty[n_begin + n0 + t], T, a.status);
                }
                s_np[t] = p;
                s_nt[t] = ty;
#pragma unroll
                for (int w = 0; w < kCW; ++w) s_nf[w][0][t] = s_nf[w][1][t] = s_nf[w][2][t] = Acc(0);
            }
            __syncthreads();
            cluster_boxes<kCJ>(s_np, mn, s_jb);
            __syncthreads();

            Acc(*nf)[kCTile] = s_nf[warp];
            for (int ic = warp; ic < nic; ic += kCW) {
                const int ia = ic * kCI + il;
                const float4 pi = s_hp[ia];
                const int tiT = s_ht[ia] * T;
                float ib[6];
#pragma unroll
                for (int d = 0; d < 6; ++d) ib[d] = s_ib[ic][d];
                Acc ax = Acc(0), ay = Acc(0), az = Acc(0);
                // on the diagonal tile only j-clusters that hold some atom after ia
                const int jc0 = diag ? (ic * kCI) / kCJ : 0;
                for (int jb = jc0; jb < njc; jb += 32) {
                    const int jt = jb + lane;
                    bool in = false;
                    if (jt < njc) {
                        const float *q = s_jb[jt];
                        const float gx = fmaxf(0.f, fmaxf(ib[0] - q[3], q[0] - ib[3]));
                        const float gy = fmaxf(0.f, fmaxf(ib[1] - q[4], q[1] - ib[4]));
                        const float gz = fmaxf(0.f, fmaxf(ib[2] - q[5], q[2] - ib[5]));
                        in = gx * gx + gy * gy + gz * gz < rc2m;
                    }
                    unsigned todo = __ballot_sync(0xffffffffu, in);
                    while (todo) {
                        const int jc = jb + __ffs(todo) - 1;
                        todo &= todo - 1;
                        const int ja = jc * kCJ + jl;
                        const float4 pj = s_np[ja];
                        const float dx = (pi.x - pj.x) + g.lo[0];
                        const float dy = (pi.y - pj.y) + g.lo[1];
                        const float dz = (pi.z - pj.z) + g.lo[2];
                        const float r2 = pair_r2(dx, dy, dz);
                        const bool ok = r2 < rc2 && ja < mn && (!diag || ia < ja);
                        const float2 ab = s_ab[tiT + s_nt[ja]];
                        const float kqq = __fmul_rn(kc, __fmul_rn(pi.w, pj.w));
                        float ir, ir2, ir6;
                        float f = pair_f(r2, ab.x, ab.y, kqq, ir, ir2, ir6);
                        f = ok ? f : 0.0f;
                        const float fx = __fmul_rn(f, dx), fy = __fmul_rn(f, dy), fz = __fmul_rn(f, dz);
                        Acc vx, vy, vz;
                        if (MODE == MD_ACCUM_FIXED64) {
                            vx = (Acc)(ok ? to_fixed(fx, a.status) : 0);
                            vy = (Acc)(ok ? to_fixed(fy, a.status) : 0);
                            vz = (Acc)(ok ? to_fixed(fz, a.status) : 0);
                        } else {
                            vx = (Acc)fx;
                            vy = (Acc)fy;
                            vz = (Acc)fz;
                        }
                        ax += vx;
                        ay += vy;
                        az += vz;
                        // reaction on ja: sum over the kCI lanes that share it
#pragma unroll
                        for (int o = 1; o < kCI; o <<= 1) {
                            vx += __shfl_xor_sync(0xffffffffu, vx, o);
                            vy += __shfl_xor_sync(0xffffffffu, vy, o);
                            vz += __shfl_xor_sync(0xffffffffu, vz, o);
                        }
                        if (il == 0) {
                            nf[0][ja] -= vx;
                            nf[1][ja] -= vy;
                            nf[2][ja] -= vz;
                        }
                        if (ok) {
                            cnt += 1;
                            if (ENERGY) {
                                e_lj += pair_u_lj(ab.x, ab.y, ir6);
                                e_c += kqq * ir;
                                vir += f * r2;
                            }
                        }
                    }
                }
                // i-forces: sum over the kCJ lanes that share ia; the i-cluster belongs
                // to this warp alone
#pragma unroll
                for (int o = kCI; o < 32; o <<= 1) {
                    ax += __shfl_xor_sync(0xffffffffu, ax, o);
                    ay += __shfl_xor_sync(0xffffffffu, ay, o);
                    az += __shfl_xor_sync(0xffffffffu, az, o);
                }
                if (jl == 0 && ia < mh) {
                    s_hf[0][ia] += ax;
                    s_hf[1][ia] += ay;
                    s_hf[2][ia] += az;
                }
            }
            __syncthreads();
            for (int t = threadIdx.x; t < mn; t += kCT) {
                Acc sx = s_nf[0][0][t], sy = s_nf[0][1][t], sz = s_nf[0][2][t];
#pragma unroll
                for (int w = 1; w < kCW; ++w) {
                    sx += s_nf[w][0][t];
                    sy += s_nf[w][1][t];
                    sz += s_nf[w][2][t];
                }
                if (diag) {
                    // the neighbour tile is the home tile: reactions join the home sums
                    s_hf[0][t] += sx;
                    s_hf[1][t] += sy;
                    s_hf[2][t] += sz;
                } else {
                    const int s = n_begin + n0 + t;
                    if (MODE == MD_ACCUM_FIXED64) {
                        unsigned long long *acc = static_cast<unsigned long long *>(a.accum);
                        atomicAdd(&acc[s], (unsigned long long)sx);
                        atomicAdd(&acc[(size_t)a.n + s], (unsigned long long)sy);
                        atomicAdd(&acc[2 * (size_t)a.n + s], (unsigned long long)sz);
                    } else {
                        red_add_v4(static_cast<float4 *>(a.accum) + s, (float)sx, (float)sy, (float)sz);
                    }
                }
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < mh; t += kCT) {
            const int s = h_begin + h0 + t;
            if (MODE == MD_ACCUM_FIXED64) {
                unsigned long long *acc = static_cast<unsigned long long *>(a.accum);
                atomicAdd(&acc[s], (unsigned long long)s_hf[0][t]);
                atomicAdd(&acc[(size_t)a.n + s], (unsigned long long)s_hf[1][t]);
                atomicAdd(&acc[2 * (size_t)a.n + s], (unsigned long long)s_hf[2][t]);
            } else {
                red_add_v4(static_cast<float4 *>(a.accum) + s, (float)s_hf[0][t], (float)s_hf[1][t],
                           (float)s_hf[2][t]);
            }
        }
    }
    block_partial<kCT>((double)e_lj, (double)e_c, (double)vir, cnt, mine);
}

// Cluster-order accumulators -> forces_out in input order.
template <int MODE>
__global__ void __launch_bounds__(256)
k_finalize_clu(const void *__restrict__ accum, const int32_t *__restrict__ corder,
               const int32_t *__restrict__ perm, int n, void *__restrict__ forces_out,
               uint32_t *status)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int o = perm[corder[s]];
    if (MODE == MD_ACCUM_FIXED64) {
        const long long *acc = static_cast<const long long *>(accum);
        long long *F = static_cast<long long *>(forces_out);
        F[3 * o + 0] = acc[s];
        F[3 * o + 1] = acc[(size_t)n + s];
        F[3 * o + 2] = acc[2 * (size_t)n + s];
    } else {
        const float4 v = static_cast<const float4 *>(accum)[s];
        float *F = static_cast<float *>(forces_out);
        F[3 * o + 0] = v.x;
        F[3 * o + 1] = v.y;
        F[3 * o + 2] = v.z;
        if (!isfinite(v.x + v.y + v.z)) set_status(status, MD_STATUS_NONFINITE);
    }
}

template <int MODE, bool ENERGY>
void launch_cluster_t(const CluArgs &c, dim3 grid, cudaStream_t stream)
{
    const size_t dyn = sizeof(float2) * (size_t)c.ntypes * (size_t)c.ntypes;
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_cluster<MODE, ENERGY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)(sizeof(float2) * kMaxTypes * kMaxTypes));
    (void)attr;
    k_cluster<MODE, ENERGY><<<grid, kCT, dyn, stream>>>(c);
}

}  // namespace

bool cluster_kernel_applies(const BoxF &box)
{
    return half_shell_pairs_per_cell(box) == 14;
}

cudaError_t launch_cluster(const ForceArgs &a, const WsLayout &ws, char *wsp, Partial *partials,
                           int *nblocks_out, cudaStream_t stream)
{
    const size_t acc_bytes = (size_t)a.n * (a.mode == MD_ACCUM_FIXED64 ? 24 : 16);
    void *accum = wsp + ws.accum;
    float4 *cpq = reinterpret_cast<float4 *>(wsp + ws.clu_pos_q);
    int32_t *cty = reinterpret_cast<int32_t *>(wsp + ws.clu_type);
    int32_t *corder = reinterpret_cast<int32_t *>(wsp + ws.clu_order);
    cudaError_t e = cudaMemsetAsync(accum, 0, acc_bytes, stream);
    if (e != cudaSuccess) return e;
    k_cluster_order<<<a.box.ncell, kOrderThreads, 0, stream>>>(a.cell_start, a.pos_q_sorted,
                                                               a.type_sorted, a.box, cpq, cty, corder);
    CluArgs c;
    c.cell_start = a.cell_start;
    c.pq = cpq;
    c.ty = cty;
    c.box = a.box;
    c.AB = a.AB;
    c.ntypes = a.ntypes;
    c.kc = a.k_coulomb;
    cutoff_thresholds(a.box, a.rc64, false, &c.rc2, &c.rc2m);
    c.accum = accum;
    c.n = a.n;
    c.partials = partials;
    c.status = a.status;
    dim3 grid(a.box.ncell, 14);
    const bool en = a.energy_virial_out != nullptr;
    const int g = (a.n + 255) / 256;
    if (a.mode == MD_ACCUM_FIXED64) {
        if (en) launch_cluster_t<MD_ACCUM_FIXED64, true>(c, grid, stream);
        else launch_cluster_t<MD_ACCUM_FIXED64, false>(c, grid, stream);
        k_finalize_clu<MD_ACCUM_FIXED64><<<g, 256, 0, stream>>>(accum, corder, a.perm, a.n, a.forces_out, a.status);
    } else {
        if (en) launch_cluster_t<MD_ACCUM_F32, true>(c, grid, stream);
        else launch_cluster_t<MD_ACCUM_F32, false>(c, grid, stream);
        k_finalize_clu<MD_ACCUM_F32><<<g, 256, 0, stream>>>(accum, corder, a.perm, a.n, a.forces_out, a.status);
    }
    *nblocks_out = a.box.ncell * 14;
    return cudaGetLastError();
}

}  // namespace mdnb
