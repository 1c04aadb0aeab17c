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
//            (alternating direction), so that consecutive atoms are neighbours.  Every
//            8 consecutive atoms of a cell form a cluster.
//   filter:  one lane per neighbour cluster tests the gap between the bounding boxes
//            of a home cluster and 32 neighbour clusters at once (rc'^2, conservative);
//            a ballot lists the clusters in range (about 37% of their 64 pairs lie
//            within rc on the dense workloads, against 14% of the cell-pair
//            candidates).
//   force:   a warp evaluates the 8 x 8 pairs of one cluster pair: lane i + 4 j holds
//            home atoms i and i + 4 and neighbour atom j and evaluates those two pairs,
//            with packed FP32x2 instructions (Blackwell's paired FP32 ALU) and the
//            exact test r^2 < rc^2 per pair.  In MD_ACCUM_FIXED64 the packed chain is
//            pair_r2 / pair_f element by element on the same staged coordinates and
//            shifts as the half-shell kernel, and every packed instruction rounds as
//            its scalar counterpart, so its integers are the same bits as the other
//            kernels'.  (pair_f ends in a fused multiply-add: a separate multiply
//            feeding an add was fused by the compiler in the packed chain only.)
//            MD_ACCUM_F32 takes k q_i once per home cluster.
//   reduce:  home-atom forces stay in registers for the whole home cluster; the
//            reaction on each neighbour atom is summed over its two pairs, then over
//            its 4 lanes by two shuffles, and added to a warp-private shared array
//            (F32) or with one integer shared atomic per component (FIXED64).
//
// Boxes with an axis of 2 cells meet each distinct stencil cell once, with unshifted
// tiles: the filter takes the gap between the clusters' nearest images and each pair
// the per-pair minimum image.  For a system alone (FP32, FIXED64) each of their few,
// long cell pairs is split over kMiSplit CTAs by home cluster.
//
// The above is the one-cluster-pair form (k_cluster), used for the fixed-point modes,
// energies, the Verlet step, batches and small grids.  FP32 forces on grids that fill the
// GPU run the long-row form (k_cluster_rows, further below): the same pairs, filter and
// pair math, but each warp takes one home cluster against all its in-range neighbour
// clusters of a group of cells, with 8 pairs a lane per step.
#include <math.h>

#include "md_internal.cuh"
#include "md_pairgeom.cuh"

namespace mdnb {
namespace {

constexpr int kCS = 8;          // atoms per cluster
constexpr int kCW = 4;          // warps per CTA
constexpr int kCT = kCW * 32;   // threads per CTA
constexpr int kCTile = 256;     // atoms of a cell staged at once (whole clusters)
constexpr int kSortMax = 1024;  // cells with more atoms keep their sorted order
constexpr int kOrderThreads = 256;
constexpr int kOrderCols = 64;   // at most 8 x 8 columns per cell

static_assert(kCTile % kCS == 0 && kCTile / kCS <= 32, "a tile's clusters fit one ballot");

// What a launch accumulates besides the forces (the partials are written only when
// asked for).
constexpr int kStatsNone = 0;    // forces only
constexpr int kStatsCount = 1;   // + within-cutoff pair count
constexpr int kStatsEnergy = 2;  // + count, energies and virial
// Per cell: sort its atoms by (column, z along the column) and write the reordered
// copies.  corder[k] is the sorted-order slot of cluster-order slot k.  The members are
// counted per column and each is ranked only against its own column's keys.  (The MD steps
// build their cells in this order directly: k_sort_cluster.)
__global__ void __launch_bounds__(kOrderThreads)
k_cluster_order(const int32_t *__restrict__ cell_start, const float4 *__restrict__ pq,
                const int32_t *__restrict__ ty, BoxF box, float4 *__restrict__ cpq,
                int32_t *__restrict__ cty, int32_t *__restrict__ corder, void *__restrict__ accum,
                int mode, int n, float4 *__restrict__ cbox)
{
    __shared__ unsigned long long s_key[kSortMax];  // by sorted slot
    __shared__ unsigned long long s_bkt[kSortMax];  // grouped by column
    __shared__ int s_col[kOrderCols + 1];           // counts, then column starts
    __shared__ int s_fill[kOrderCols];
    pdl_trigger();  // the force kernel may be scheduled now; it waits for this pass
    const int cg = blockIdx.x, c = cg;
    const int b = cell_start[cg], m = cell_start[cg + 1] - b;
    if (m <= 0) return;
    // the force kernel's accumulators of this cell's slots start at zero
    for (int t = threadIdx.x; t < m; t += kOrderThreads) {
        if (fixed_output(mode)) {
            unsigned long long *A = static_cast<unsigned long long *>(accum);
            A[b + t] = 0ull;
            A[(size_t)n + b + t] = 0ull;
            A[2 * (size_t)n + b + t] = 0ull;
        } else {
            static_cast<float4 *>(accum)[b + t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
    if (m > kSortMax) {
        for (int t = threadIdx.x; t < m; t += kOrderThreads) {
            corder[b + t] = b + t;
            cpq[b + t] = pq[b + t];
            cty[b + t] = ty[b + t];
        }
        __syncthreads();
        write_cluster_boxes<kOrderThreads>(cpq + b, b, m, cbox, n);
        return;
    }
    const int nx = box.dims[0], ny = box.dims[1];
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    // about 20 atoms per column
    const int S = max(1, min(8, (int)(sqrtf((float)m * (1.0f / 20.0f)) + 0.5f)));
    const int ncol = S * S;
    for (int t = threadIdx.x; t < ncol; t += kOrderThreads) {
        s_col[t] = 0;
        s_fill[t] = 0;
    }
    __syncthreads();
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
    for (int t = threadIdx.x; t < m; t += kOrderThreads) {
        const unsigned long long k = s_key[t];
        const int col = (int)(k >> 44);
        s_bkt[s_col[col] + atomicAdd(&s_fill[col], 1)] = k;
    }
    __syncthreads();
    // each member ranked against its own column only
    for (int t = threadIdx.x; t < m; t += kOrderThreads) {
        const unsigned long long k = s_key[t];
        const int col = (int)(k >> 44);
        const int b0 = s_col[col], b1 = s_col[col + 1];
        int rank = b0;
        for (int u = b0; u < b1; ++u) rank += s_bkt[u] < k;
        corder[b + rank] = b + t;
        cpq[b + rank] = pq[b + t];
        cty[b + rank] = ty[b + t];
    }
    __syncthreads();
    write_cluster_boxes<kOrderThreads>(cpq + b, b, m, cbox, n);
}

// Packed pairs of FP32 values (element 0 in the low half).
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2_make(float lo, float hi)
{
    f2 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ void f2_split(f2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
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
    // Verlet step (GATHER): slot s holds atom perm[s]; its current position is gpq[perm[s]]
    // (input order, wrapped in FP64 and rounded to float)
    const float4 *gpq;
    const int32_t *perm;
    // cluster boxes of the cluster-ordered arrays (long-row form), or null
    const float4 *cbox;
};

// Bounding boxes of the clusters of a staged tile (padding excluded).
__device__ __forceinline__ void cluster_boxes(const float4 *p, int m, float (*box)[kCTile / kCS])
{
    const int nclu = (m + kCS - 1) / kCS;
    for (int k = threadIdx.x; k < nclu; k += kCT) {
        float lo[3] = {kFar, kFar, kFar}, hi[3] = {-kFar, -kFar, -kFar};
        const int e = min(m, (k + 1) * kCS);
        for (int t = k * kCS; t < e; ++t) {
            const float4 q = p[t];
            lo[0] = fminf(lo[0], q.x); hi[0] = fmaxf(hi[0], q.x);
            lo[1] = fminf(lo[1], q.y); hi[1] = fmaxf(hi[1], q.y);
            lo[2] = fminf(lo[2], q.z); hi[2] = fmaxf(hi[2], q.z);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            box[d][k] = lo[d];
            box[d + 3][k] = hi[d];
        }
    }
}

// Shared tiles of one CTA.  Reactions: F32 one array per warp (plain read-modify-write,
// no float atomics); FIXED64 one array for the CTA (native integer shared atomics).
// Home forces need no array: each home cluster's sums go to global memory per row.
template <int MODE>
struct CluSmem {
    using Acc = typename AccT<MODE>::T;
    static constexpr int NW = MODE == MD_ACCUM_FIXED64 ? 1 : kCW;
    float4 hp[kCTile];  // home tile (x, y, z shifted, q)
    float4 np[kCTile];  // neighbour tile
    unsigned char ht[kCTile], nt[kCTile];  // LJ types (below kMaxTypes = 32)
    float ib[6][kCTile / kCS];  // home cluster boxes: lo xyz, hi xyz (one row per bound)
    float jb[6][kCTile / kCS];  // neighbour cluster boxes
    // reactions on neighbour atoms (this tile), component d of atom t at d * kRow + t;
    // F32 rows are 8 words longer, so that the three lanes that add the x, y and z of
    // one atom hit different banks
    static constexpr int kRow = kCTile + (MODE == MD_ACCUM_FIXED64 ? 0 : 8);
    Acc nf[NW][2 * kRow + kCTile];
    __device__ __forceinline__ Acc &react(int w, int d, int t) { return nf[w][d * kRow + t]; }
    int next;                   // next home cluster to hand out
    // Verlet step: one bit per tile atom whose coordinate was wrapped across a face of
    // the box since the cells were built (home and neighbour tile)
    unsigned hwb[kCTile / 32], jwb[kCTile / 32];
};

struct CluConst {
    void *accum;  // cluster-order accumulators (global); home sums go there per row
    int n, hbase; // atoms; slot of the home tile's first atom
    float kc, rc2, rc2m;
    float lo[3];
    float hs[3], ns[3];  // the cell pair's shifts of home and neighbour coordinates
    float L[3], Lhi[3], Llo[3], invL[3];  // per-pair minimum image (boxes with a 2-cell axis)
    int T;
    uint32_t *status;
};

// Verlet step: whether cluster c of a tile holds an atom wrapped since the cells were
// built (the 8 bits of its atoms in the tile's mask).
__device__ __forceinline__ bool wrapped_cluster(const unsigned *bits, int c)
{
    return ((bits[c >> 2] >> ((c & 3) * 8)) & 0xffu) != 0u;
}
__device__ __forceinline__ bool wrapped_atom(const unsigned *bits, int t)
{
    return ((bits[t >> 5] >> (t & 31)) & 1u) != 0u;
}

// Home cluster ic against every neighbour cluster of the staged tile in range.
// DIAG: the neighbour tile is the home tile (pairs ia < ja only); SHIFT: the cell
// pair has a remainder shift to add to the difference; MI: the per-pair minimum image
// (boxes with an axis of 2 cells, unshifted tiles).  GATHER (Verlet step, boxes with >= 3
// cells per axis): a cluster pair with an atom wrapped across a face of the box since the
// cells were built passes the box filter and takes the per-pair minimum image of the
// unshifted coordinates (staged + shift, exact), which for a pair within rc gives the
// bits of the shifted difference the plain step forms from freshly built cells.
template <int MODE, int STATS, bool DIAG, bool SHIFT, bool MI, bool GATHER = false>
__device__ __forceinline__ void cluster_row(CluSmem<MODE> &sm, const float2 *s_ab,
                                            const CluConst &k, int ic, int njc, int mh, int warp,
                                            int lane, float &e_lj, float &e_c, float &vir,
                                            unsigned &cnt)
{
    using Acc = typename AccT<MODE>::T;
    const int il = lane & 3, jl = lane >> 2;
    const int ia0 = ic * kCS + il, ia1 = ia0 + 4;
    const float4 p0 = sm.hp[ia0], p1 = sm.hp[ia1];
    const bool hrow_wr = GATHER && wrapped_cluster(sm.hwb, ic);
    const f2 xi = f2_make(p0.x, p1.x), yi = f2_make(p0.y, p1.y), zi = f2_make(p0.z, p1.z);
    const f2 qi = f2_make(p0.w, p1.w);
    const int t0 = sm.ht[ia0] * k.T, t1 = sm.ht[ia1] * k.T;
    const f2 kc2 = f2_make(k.kc, k.kc);
    const f2 kcq = f2_mul(kc2, qi);  // k q_i (F32 path)
    const f2 lox = f2_make(k.lo[0], k.lo[0]), loy = f2_make(k.lo[1], k.lo[1]),
             loz = f2_make(k.lo[2], k.lo[2]);
    float ib[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) ib[d] = sm.ib[d][ic];
    // MI: the box filter takes the gap between the clusters' nearest images, from their
    // centres and half extents (widened by a few ulps of L for the roundings)
    float ic_c[3], ic_e[3];
    if (MI) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            ic_c[d] = 0.5f * (ib[d] + ib[d + 3]);
            ic_e[d] = 0.5f * (ib[d + 3] - ib[d]) + 4.0f * 1.1920929e-7f * k.L[d];
        }
    }
    // home-atom sums: F32 packed (atom ia0 low, ia1 high); FIXED64 one integer each
    f2 ax2 = 0ull, ay2 = 0ull, az2 = 0ull;
    Acc ax0 = Acc(0), ay0 = Acc(0), az0 = Acc(0), ax1 = Acc(0), ay1 = Acc(0), az1 = Acc(0);

    const int jc0 = DIAG ? ic : 0;
    for (int jb = jc0; jb < njc; jb += 32) {
        const int jt = jb + lane;
        bool in = false;
        if (jt < njc) {
            if (MI) {
                float g2 = 0.f;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float jcen = 0.5f * (sm.jb[d][jt] + sm.jb[d + 3][jt]);
                    const float jext = 0.5f * (sm.jb[d + 3][jt] - sm.jb[d][jt]);
                    float dd = ic_c[d] - jcen;
                    dd -= k.L[d] * rintf(dd * k.invL[d]);
                    const float gap = fmaxf(0.f, fabsf(dd) - ic_e[d] - jext);
                    g2 += gap * gap;
                }
                in = g2 < k.rc2m;
            } else {
                const float gx = fmaxf(0.f, fmaxf(ib[0] - sm.jb[3][jt], sm.jb[0][jt] - ib[3]));
                const float gy = fmaxf(0.f, fmaxf(ib[1] - sm.jb[4][jt], sm.jb[1][jt] - ib[4]));
                const float gz = fmaxf(0.f, fmaxf(ib[2] - sm.jb[5][jt], sm.jb[2][jt] - ib[5]));
                in = gx * gx + gy * gy + gz * gz < k.rc2m;
                // a cluster with a wrapped atom has no meaningful box here: always a candidate
                if (GATHER && (hrow_wr || wrapped_cluster(sm.jwb, jt))) in = true;
            }
        }
        unsigned todo = __ballot_sync(0xffffffffu, in);
        while (todo) {
            const int jc = jb + __ffs(todo) - 1;
            todo &= todo - 1;
            const int ja = jc * kCS + jl;
            const float4 pj = sm.np[ja];
            const int tj = sm.nt[ja];
            const float2 ab0 = s_ab[t0 + tj], ab1 = s_ab[t1 + tj];  // (A, -B)
            // pair_r2 and pair_f element by element in packed FP32x2 instructions
            // (each rounds as its scalar counterpart)
            f2 dx, dy, dz;
            if (MI) {
                // the library's per-pair minimum image, element by element
                dx = f2_make(min_image_f32(p0.x, pj.x, k.Lhi[0], k.Llo[0], k.invL[0]),
                             min_image_f32(p1.x, pj.x, k.Lhi[0], k.Llo[0], k.invL[0]));
                dy = f2_make(min_image_f32(p0.y, pj.y, k.Lhi[1], k.Llo[1], k.invL[1]),
                             min_image_f32(p1.y, pj.y, k.Lhi[1], k.Llo[1], k.invL[1]));
                dz = f2_make(min_image_f32(p0.z, pj.z, k.Lhi[2], k.Llo[2], k.invL[2]),
                             min_image_f32(p1.z, pj.z, k.Lhi[2], k.Llo[2], k.invL[2]));
            } else if (GATHER && (hrow_wr || wrapped_cluster(sm.jwb, jc))) {
                // the unshifted coordinates: a wrapped atom was staged as it is, any
                // other with the cell pair's shift subtracted (exactly), so adding it back
                // restores the coordinate exactly
                const bool w0 = wrapped_atom(sm.hwb, ia0), w1 = wrapped_atom(sm.hwb, ia1);
                const bool wj = wrapped_atom(sm.jwb, ja);
                float r0[3] = {p0.x, p0.y, p0.z}, r1[3] = {p1.x, p1.y, p1.z}, rj[3] = {pj.x, pj.y, pj.z};
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (!w0) r0[d] = __fadd_rn(r0[d], k.hs[d]);
                    if (!w1) r1[d] = __fadd_rn(r1[d], k.hs[d]);
                    if (!wj) rj[d] = __fadd_rn(rj[d], k.ns[d]);
                }
                dx = f2_make(min_image_f32(r0[0], rj[0], k.Lhi[0], k.Llo[0], k.invL[0]),
                             min_image_f32(r1[0], rj[0], k.Lhi[0], k.Llo[0], k.invL[0]));
                dy = f2_make(min_image_f32(r0[1], rj[1], k.Lhi[1], k.Llo[1], k.invL[1]),
                             min_image_f32(r1[1], rj[1], k.Lhi[1], k.Llo[1], k.invL[1]));
                dz = f2_make(min_image_f32(r0[2], rj[2], k.Lhi[2], k.Llo[2], k.invL[2]),
                             min_image_f32(r1[2], rj[2], k.Lhi[2], k.Llo[2], k.invL[2]));
            } else {
                dx = f2_sub(xi, f2_dup(pj.x));
                dy = f2_sub(yi, f2_dup(pj.y));
                dz = f2_sub(zi, f2_dup(pj.z));
                if (SHIFT) {
                    dx = f2_add(dx, lox);
                    dy = f2_add(dy, loy);
                    dz = f2_add(dz, loz);
                }
            }
            const f2 r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
            float r20, r21;
            f2_split(r2, r20, r21);
            // padding sits at +-1e18: such pairs fail the cutoff test
            const bool ok0 = r20 < k.rc2 && (!DIAG || ia0 < ja);
            const bool ok1 = r21 < k.rc2 && (!DIAG || ia1 < ja);
            const f2 A2 = f2_make(ab0.x, ab1.x), nB2 = f2_make(ab0.y, ab1.y);
            // FIXED64 keeps the library's k (q_i q_j) so that its integers match the
            // other kernels; F32 uses (k q_i) q_j
            const f2 kqq = MODE == MD_ACCUM_FIXED64 ? f2_mul(kc2, f2_mul(qi, f2_dup(pj.w)))
                                                    : f2_mul(kcq, f2_dup(pj.w));
            float y0, y1;
            y0 = rsqrt_hw(r20);
            y1 = rsqrt_hw(r21);
            const f2 y = f2_make(y0, y1);
            const f2 ir = y;
            const f2 ir2 = f2_mul(ir, ir);
            const f2 ir6 = f2_mul(f2_mul(ir2, ir2), ir2);
            const f2 ir8 = f2_mul(ir6, ir2);
            const f2 lj = f2_mul(ir8, f2_fma(A2, ir6, nB2));
            float f0, f1;
            f2_split(f2_fma(f2_mul(kqq, ir2), ir, lj), f0, f1);
            f0 = ok0 ? f0 : 0.0f;
            f1 = ok1 ? f1 : 0.0f;
            const f2 f = f2_make(f0, f1);
            const f2 fx = f2_mul(f, dx), fy = f2_mul(f, dy), fz = f2_mul(f, dz);
            Acc vx, vy, vz;  // reaction on ja (before the sign): this lane's two pairs
            if (MODE == MD_ACCUM_FIXED64) {
                float x0, x1, y0_, y1_, z0, z1;
                f2_split(fx, x0, x1);
                f2_split(fy, y0_, y1_);
                f2_split(fz, z0, z1);
                const Acc gx0 = (Acc)(ok0 ? to_fixed(x0, k.status) : 0), gx1 = (Acc)(ok1 ? to_fixed(x1, k.status) : 0);
                const Acc gy0 = (Acc)(ok0 ? to_fixed(y0_, k.status) : 0), gy1 = (Acc)(ok1 ? to_fixed(y1_, k.status) : 0);
                const Acc gz0 = (Acc)(ok0 ? to_fixed(z0, k.status) : 0), gz1 = (Acc)(ok1 ? to_fixed(z1, k.status) : 0);
                ax0 += gx0; ay0 += gy0; az0 += gz0;
                ax1 += gx1; ay1 += gy1; az1 += gz1;
                vx = gx0 + gx1;
                vy = gy0 + gy1;
                vz = gz0 + gz1;
            } else {
                ax2 = f2_add(ax2, fx);
                ay2 = f2_add(ay2, fy);
                az2 = f2_add(az2, fz);
                float a0, a1;
                f2_split(fx, a0, a1);
                vx = (Acc)(a0 + a1);
                f2_split(fy, a0, a1);
                vy = (Acc)(a0 + a1);
                f2_split(fz, a0, a1);
                vz = (Acc)(a0 + a1);
            }
            if (STATS >= kStatsCount) cnt += (unsigned)ok0 + (unsigned)ok1;
            if (STATS == kStatsEnergy) {
                float i6a, i6b, ira, irb, ka, kb;
                f2_split(ir6, i6a, i6b);
                f2_split(ir, ira, irb);
                f2_split(kqq, ka, kb);
                if (ok0) {
                    e_lj += pair_u_lj(ab0.x, -ab0.y, i6a);
                    e_c += ka * ira;
                    vir += f0 * r20;
                }
                if (ok1) {
                    e_lj += pair_u_lj(ab1.x, -ab1.y, i6b);
                    e_c += kb * irb;
                    vir += f1 * r21;
                }
            }
            {
                // reduce-scatter of (x, y, z, 0) over the 4 lanes of ja (3 shuffles instead
                // of the 6 of a butterfly): the lanes with il & 2 keep (z, 0), the others
                // (x, y); then il & 1 picks one of the two.  Lane il ends with component il.
                const bool hi2 = (il & 2) != 0, hi1 = (il & 1) != 0;
                const Acc s0 = hi2 ? vx : vz, s1 = hi2 ? vy : Acc(0);
                const Acc k0 = (hi2 ? vz : vx) + __shfl_xor_sync(0xffffffffu, s0, 2);
                const Acc k1 = (hi2 ? Acc(0) : vy) + __shfl_xor_sync(0xffffffffu, s1, 2);
                const Acc t = (hi1 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, hi1 ? k0 : k1, 1);
                if (il < 3) {
                    if (MODE == MD_ACCUM_FIXED64)
                        atomicAdd(reinterpret_cast<unsigned long long *>(&sm.react(0, il, ja)), (unsigned long long)(Acc(0) - t));
                    else
                        sm.react(warp, il, ja) -= t;
                }
            }
        }
    }
    // home-atom sums over the 8 lanes that share them (the home cluster belongs to this
    // warp alone within the CTA): a reduce-scatter of the six (atom, component) sums over
    // the lane bits of jl, after which lane jl < 6 holds sum jl (atom ia0 for jl < 3,
    // ia1 above, component jl % 3) and adds it to the global accumulator (a home
    // cluster meets each neighbour tile once, so there is nothing to gather in shared
    // memory first)
    if (MODE != MD_ACCUM_FIXED64) {
        float a, b;
        f2_split(ax2, a, b);
        ax0 = (Acc)a;
        ax1 = (Acc)b;
        f2_split(ay2, a, b);
        ay0 = (Acc)a;
        ay1 = (Acc)b;
        f2_split(az2, a, b);
        az0 = (Acc)a;
        az1 = (Acc)b;
    }
    Acc w[8] = {ax0, ay0, az0, ax1, ay1, az1, Acc(0), Acc(0)};
#pragma unroll
    for (int half = 4, o = 16; half >= 1; half >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;  // keep the upper half of the current values
#pragma unroll
        for (int q = 0; q < half; ++q) {
            const Acc send = up ? w[q] : w[q + half];
            const Acc keep = up ? w[q + half] : w[q];
            w[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    if (jl < 6) {
        const int ia = jl < 3 ? ia0 : ia1;
        if (ia < mh) {
            const size_t s = (size_t)(k.hbase + ia);
            const int d = jl < 3 ? jl : jl - 3;
            if (MODE == MD_ACCUM_FIXED64)
                atomicAdd(static_cast<unsigned long long *>(k.accum) + (size_t)d * k.n + s,
                          (unsigned long long)w[0]);
            else if (MODE == MD_ACCUM_FIXED_TILE)  // this row's sum, rounded once
                atomicAdd(static_cast<unsigned long long *>(k.accum) + (size_t)d * k.n + s,
                          (unsigned long long)to_fixed((float)w[0], k.status));
            else
                atomicAdd(static_cast<float *>(k.accum) + 4 * s + d, (float)w[0]);
        }
    }
}

// Verlet step: whether a staged coordinate lies on the far side of the box from the
// centre of the cell its atom was binned into (it crossed a face since the cells were
// built; an atom that has not moves less than half a box from its cell).
__device__ __forceinline__ bool crossed_face(const float4 &p, const float *centre, const float *half_L)
{
    return fabsf(p.x - centre[0]) > half_L[0] || fabsf(p.y - centre[1]) > half_L[1] ||
           fabsf(p.z - centre[2]) > half_L[2];
}

// One cell pair: cell cx of the launch (of gx) with stencil entry cy (of gy), or the
// share z of zs of its home clusters (rows z, z + zs, ...: boxes with an axis of 2 cells
// split each cell pair over kMiSplit CTAs, whose few cell pairs are long).
template <int MODE, int STATS, bool BATCHED, bool MI, bool GATHER = false>
__device__ __forceinline__ void cluster_item(CluSmem<MODE> &sm, float2 *s_ab, const CluArgs &a,
                                             const BatchArgs &bt,
                                             unsigned long long *sys_pair_count, int cx, int cy,
                                             int gx, int z = 0, int zs = 1, int gy = 1)
{
    using Acc = typename AccT<MODE>::T;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float e_lj = 0.f, e_c = 0.f, vir = 0.f;
    unsigned cnt = 0;
    Partial *mine = a.partials + ((size_t)z * gy + cy) * gx;

    // the system this CTA works on: the only one, or the one its cell belongs to
    PairGeom g;
    CluConst k;
    const float2 *AB;
    bool valid;
    int sid = 0;
    if (BATCHED) {
        // regular systems' cells first in cell_list, then those with a 2-cell axis
        const int cell = bt.cell_list[(MI ? bt.ncell_reg : 0) + cx];
        sid = bt.cell_sys[cell];
        const SysDesc &d = bt.sys[sid];
        valid = cell_pair(d.box, cell - d.cell_offset, cy, g);
        if (MI) {
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                k.L[e] = (float)d.box.L[e];
                k.Lhi[e] = d.box.Lhi[e];
                k.Llo[e] = d.box.Llo[e];
                k.invL[e] = d.box.invL[e];
            }
        }
        g.home += d.cell_offset;
        g.nbr += d.cell_offset;
        k.T = d.ntypes;
        AB = d.AB;
        k.kc = d.kc;
        k.rc2 = d.rc2;
        k.rc2m = d.rc2m;
    } else {
        valid = cell_pair(a.box, cx, cy, g);
        if (MI || GATHER) {
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                k.L[e] = (float)a.box.L[e];
                k.Lhi[e] = a.box.Lhi[e];
                k.Llo[e] = a.box.Llo[e];
                k.invL[e] = a.box.invL[e];
            }
        }
        k.T = a.ntypes;
        AB = a.AB;
        k.kc = a.kc;
        k.rc2 = a.rc2;
        k.rc2m = a.rc2m;
    }
    if (!valid) {
        if (STATS != kStatsNone) block_partial_to<kCT>(0.0, 0.0, 0.0, 0ull, mine + cx);
        return;
    }
    const int h_begin = a.cell_start[g.home], nh = a.cell_start[g.home + 1] - h_begin;
    const int n_begin = a.cell_start[g.nbr], nn = a.cell_start[g.nbr + 1] - n_begin;
    if (nh == 0 || nn == 0) {
        if (STATS != kStatsNone) block_partial_to<kCT>(0.0, 0.0, 0.0, 0ull, mine + cx);
        return;
    }
    k.status = a.status;
    k.accum = a.accum;
    k.n = a.n;
    bool shift = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        k.lo[d] = g.lo[d];
        k.hs[d] = g.hs[d];
        k.ns[d] = g.ns[d];
        shift |= g.lo[d] != 0.0f;
    }
    // Verlet step: centres of the two cells and half the box, for the face-crossing test
    float hcen[3] = {0.f, 0.f, 0.f}, ncen[3] = {0.f, 0.f, 0.f}, half_L[3] = {0.f, 0.f, 0.f};
    if (GATHER && !MI) {
        const int nx = a.box.dims[0], ny = a.box.dims[1];
        const int hc[3] = {g.home % nx, (g.home / nx) % ny, g.home / (nx * ny)};
        const int nc[3] = {g.nbr % nx, (g.nbr / nx) % ny, g.nbr / (nx * ny)};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float edge = (float)(a.box.L[d] / a.box.dims[d]);
            hcen[d] = ((float)hc[d] + 0.5f) * edge;
            ncen[d] = ((float)nc[d] + 0.5f) * edge;
            half_L[d] = 0.5f * a.box.Lhi[d];
        }
    }
    for (int t = threadIdx.x; t < k.T * k.T; t += kCT) {
        const float2 ab = AB[t];
        s_ab[t] = make_float2(ab.x, -ab.y);
    }

    for (int h0 = 0; h0 < nh; h0 += kCTile) {
        const int mh = min(kCTile, nh - h0);
        k.hbase = h_begin + h0;
        const int nic = (mh + kCS - 1) / kCS;
        __syncthreads();
        // (every thread makes the same number of passes, so that the GATHER form's ballot
        // sees whole warps)
        for (int t0 = 0; t0 < (GATHER ? kCTile : nic * kCS); t0 += kCT) {
            const int t = t0 + threadIdx.x;
            bool wr = false;
            if (t < nic * kCS) {
                float4 p;
                int ty = 0;
                if (t < mh) {
                    const int slot = h_begin + h0 + t;
                    p = GATHER ? wrap_pos_f(a.gpq[a.perm[slot]], a.box) : a.pq[slot];
                    wr = GATHER && !MI && crossed_face(p, hcen, half_L);
                    if (!wr) {  // a wrapped atom is staged as it is
                        p.x -= g.hs[0];
                        p.y -= g.hs[1];
                        p.z -= g.hs[2];
                    }
                    ty = clamp_type(a.ty[slot], k.T, a.status);
                } else {
                    p = make_float4(kFar, kFar, kFar, 0.f);
                }
                sm.hp[t] = p;
                sm.ht[t] = (unsigned char)ty;
            }
            if (GATHER) {
                const unsigned bits = __ballot_sync(0xffffffffu, wr);
                if ((threadIdx.x & 31) == 0) sm.hwb[t >> 5] = bits;
            }
        }
        __syncthreads();
        cluster_boxes(sm.hp, mh, sm.ib);
        for (int n0 = g.self ? h0 : 0; n0 < nn; n0 += kCTile) {
            const int mn = min(kCTile, nn - n0);
            const int njc = (mn + kCS - 1) / kCS;
            const bool diag = g.self && n0 == h0;
            __syncthreads();
            for (int t0 = 0; t0 < (GATHER ? kCTile : njc * kCS); t0 += kCT) {
                const int t = t0 + threadIdx.x;
                bool wr = false;
                if (t < njc * kCS) {
                    float4 p;
                    int ty = 0;
                    if (t >= mn) {
                        p = make_float4(-kFar, -kFar, -kFar, 0.f);
                    } else if (diag) {
                        p = sm.hp[t];  // the home tile holds the same atoms
                        ty = sm.ht[t];
                        wr = GATHER && wrapped_atom(sm.hwb, t);
                    } else {
                        const int slot = n_begin + n0 + t;
                        p = GATHER ? wrap_pos_f(a.gpq[a.perm[slot]], a.box) : a.pq[slot];
                        wr = GATHER && !MI && crossed_face(p, ncen, half_L);
                        if (!wr) {
                            p.x -= g.ns[0];
                            p.y -= g.ns[1];
                            p.z -= g.ns[2];
                        }
                        ty = clamp_type(a.ty[slot], k.T, a.status);
                    }
                    sm.np[t] = p;
                    sm.nt[t] = (unsigned char)ty;
#pragma unroll
                    for (int w = 0; w < CluSmem<MODE>::NW; ++w) sm.react(w, 0, t) = sm.react(w, 1, t) = sm.react(w, 2, t) = Acc(0);
                }
                if (GATHER) {
                    const unsigned bits = __ballot_sync(0xffffffffu, wr);
                    if ((threadIdx.x & 31) == 0) sm.jwb[t >> 5] = bits;
                }
            }
            __syncthreads();
            cluster_boxes(sm.np, mn, sm.jb);
            if (threadIdx.x == 0) sm.next = kCW;
            __syncthreads();
            // home clusters handed out one at a time, so that warps finish together;
            // MD_ACCUM_FIXED_TILE deals them in a fixed order (warp w takes w, w + kCW, ...)
            // so that every warp-private partial sum is formed in the same order each run
            // (this CTA's rows: home clusters z, z + zs, ...)
            const int nrow = nic > z ? (nic - z + zs - 1) / zs : 0;
            for (int r = warp; r < nrow;) {
                const int ic = r * zs + z;
                if (diag)
                    cluster_row<MODE, STATS, true, false, MI, GATHER>(sm, s_ab, k, ic, njc, mh, warp, lane, e_lj, e_c, vir, cnt);
                else if (!MI && shift)
                    cluster_row<MODE, STATS, false, true, false, GATHER>(sm, s_ab, k, ic, njc, mh, warp, lane, e_lj, e_c, vir, cnt);
                else
                    cluster_row<MODE, STATS, false, false, MI, GATHER>(sm, s_ab, k, ic, njc, mh, warp, lane, e_lj, e_c, vir, cnt);
                if (MODE == MD_ACCUM_FIXED_TILE) {
                    r += kCW;
                } else {
                    int nx = 0;
                    if (lane == 0) nx = atomicAdd(&sm.next, 1);
                    r = __shfl_sync(0xffffffffu, nx, 0);
                }
            }
            __syncthreads();
            for (int t = threadIdx.x; t < mn; t += kCT) {
                Acc sx = sm.react(0, 0, t), sy = sm.react(0, 1, t), sz = sm.react(0, 2, t);
#pragma unroll
                for (int w = 1; w < CluSmem<MODE>::NW; ++w) {
                    sx += sm.react(w, 0, t);
                    sy += sm.react(w, 1, t);
                    sz += sm.react(w, 2, t);
                }
                {
                    const int s = n_begin + n0 + t;
                    if (MODE == MD_ACCUM_FIXED64) {
                        unsigned long long *acc = static_cast<unsigned long long *>(a.accum);
                        atomicAdd(&acc[s], (unsigned long long)sx);
                        atomicAdd(&acc[(size_t)a.n + s], (unsigned long long)sy);
                        atomicAdd(&acc[2 * (size_t)a.n + s], (unsigned long long)sz);
                    } else if (MODE == MD_ACCUM_FIXED_TILE) {
                        // the tile's reaction on this atom (warps summed in a fixed
                        // order), rounded once
                        unsigned long long *acc = static_cast<unsigned long long *>(a.accum);
                        atomicAdd(&acc[s], (unsigned long long)to_fixed((float)sx, a.status));
                        atomicAdd(&acc[(size_t)a.n + s], (unsigned long long)to_fixed((float)sy, a.status));
                        atomicAdd(&acc[2 * (size_t)a.n + s], (unsigned long long)to_fixed((float)sz, a.status));
                    } else {
                        red_add_v4(static_cast<float4 *>(a.accum) + s, (float)sx, (float)sy, (float)sz);
                    }
                }
            }
        }
    }
    if (STATS != kStatsNone) {
        block_partial_to<kCT>((double)e_lj, (double)e_c, (double)vir, (unsigned long long)cnt, mine + cx);
        if (BATCHED && sys_pair_count && threadIdx.x == 0 && mine[cx].count)
            atomicAdd(&sys_pair_count[sid], mine[cx].count);
    }
}

// One CTA per cell pair (grid cells x stencil entries), or PERSIST: a grid of about one
// wave whose CTAs take cell pairs from a counter until none are left (`work`, zeroed
// before the launch; items ordered stencil entry-major like the plain grid).
// Register budget: 8 CTAs per SM (64 registers a thread), which the force, step and
// pair-counting forms fit without spilling; the FP32 force and step form takes 9 (56
// registers, and its shared memory fits 9 as well).  Summing energies carries more live
// values (7 CTAs for FP32, 6 for FIXED64), and so does the persistent FIXED64 counting
// form (6).
template <int MODE, int STATS, bool PERSIST>
constexpr int clu_min_blocks()
{
    return STATS == kStatsEnergy ? (MODE == MD_ACCUM_FIXED64 ? 6 : 7)
         : (MODE == MD_ACCUM_FIXED64 && STATS != kStatsNone && PERSIST) ? 6
         : (MODE != MD_ACCUM_FIXED64 && STATS == kStatsNone) ? 9 : 8;
}

template <int MODE, int STATS, bool BATCHED, bool MI, bool PERSIST, bool GATHER = false>
__global__ void __launch_bounds__(kCT, (clu_min_blocks<MODE, STATS, PERSIST>()))
k_cluster(CluArgs a, BatchArgs bt, unsigned long long *sys_pair_count, int *work, int ncells,
          int per_cell, int zsplit)
{
    __shared__ __align__(16) CluSmem<MODE> sm;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    float2 *s_ab = reinterpret_cast<float2 *>(s_dyn);  // LJ table [ntypes * ntypes]: (A, -B)
    pdl_wait();
    pdl_trigger();
    if (!PERSIST) {
        cluster_item<MODE, STATS, BATCHED, MI, GATHER>(sm, s_ab, a, bt, sys_pair_count, blockIdx.x,
                                                       blockIdx.y, gridDim.x, blockIdx.z, gridDim.z,
                                                       gridDim.y);
        return;
    }
    __shared__ int s_item;
    const int nitems = ncells * per_cell * zsplit;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(work, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nitems) break;
        const int pair = item % (ncells * per_cell);
        cluster_item<MODE, STATS, BATCHED, MI>(sm, s_ab, a, bt, sys_pair_count, pair % ncells,
                                               pair / ncells, ncells, item / (ncells * per_cell),
                                               zsplit, per_cell);
    }
}

// ---------------------------------------------------------------------------------------
// Long-row form of the cluster-pair kernel (MD_ACCUM_F32, boxes with >= 3 cells per
// axis, forces with or without the pair count).
//
// One CTA per (home cell, group of half-shell entries).  The group's cells (at most
// kRowCells, each at most kRowCellAtoms atoms) are staged once, and every home cluster
// of the cell is one row: its in-range neighbour clusters across all the group's cells,
// four per warp step.  Lane (slot = lane / 8, neighbour atom jl = lane % 8) holds one
// neighbour atom and evaluates it against all 8 home atoms, which every lane keeps in
// registers as packed pairs of atoms.  The reaction on the neighbour atom is therefore
// summed in registers (one vector reduction into the accumulator per step) and the home
// sums stay in registers for the whole row (one reduction over the warp per row).  The
// per-step overhead of the one-cluster-pair step is spread over 8 pairs a lane instead
// of 2.  Cells with more atoms than a tile holds make the CTA run the one-cluster-pair
// code for each of its group's entries instead.
//
// The displacement is formed exactly as in the one-cluster-pair form: neighbour tiles
// staged with ns subtracted, home coordinates with hs subtracted, lo added to the
// difference.  The group's cells are taken in classes of equal wrap code (equal hs, ns
// and lo), each class one list per row.
constexpr int kRW = 4;                 // warps per CTA
constexpr int kRT = kRW * 32;
constexpr int kRowCells = 4;           // cells per group at most
constexpr int kRowCellAtoms = 256;     // atoms per cell at most (32 clusters)
constexpr int kRowClu = kRowCells * (kRowCellAtoms / kCS);  // staged clusters at most
constexpr int kRowDummy = kRowClu;     // a cluster of padding atoms, for partial steps
constexpr int kRowSlots = (kRowClu + 1) * kCS;
constexpr int kRowList = kRowClu + 8;  // diagonal entry + padding for the last step and the prefetch
constexpr int kRowABStride = 5;        // float4 per neighbour type in a row's LJ table
constexpr int kRedRow = 25;            // floats per lane in the row-end reduction (24 + 1 pad)

// Half-shell entries (0: the cell itself; j: forward neighbour j) of the four groups,
// heaviest group first (about 840, 760, 760 and 510 cluster pairs in range at the
// lattice density: face neighbours about 390, the cell itself 310, edges 185, corners 70).
__constant__ int kRowGroup[4][kRowCells] = {{0, 1, 5, 7}, {3, 2, 4, -1}, {9, 6, 8, -1},
                                            {10, 12, 11, 13}};
constexpr int kRowGroups = 4;
// slot of entry e in kPairOrder (the one-cluster-pair grid's blockIdx.y of that pair)
__constant__ int kEntrySlot[14] = {3, 0, 4, 1, 5, 10, 6, 11, 7, 2, 8, 12, 9, 13};

struct RowSmem {
    float4 np[kRowSlots];                 // neighbour atoms (ns subtracted, q); padding -far
    int ng[kRowSlots];                    // their slots in the accumulators; -1 for padding
    float4 nlo[kRowClu], nhi[kRowClu];    // neighbour cluster boxes (padding excluded)
    float4 hp[kRowCellAtoms];             // home atoms as stored; padding +far
    float4 hlo[kRowCellAtoms / kCS], hhi[kRowCellAtoms / kCS];
    unsigned short lst[kRW][kRowList];    // per-warp list of a row's clusters in range
    unsigned char nt[kRowSlots];
    unsigned char ht[kRowCellAtoms];
    int ncl, nclass, self_nclu, next;
    int cbeg[kRowCells + 1];              // first staged cluster of each cell (class order; unused cells empty)
    int gbeg[kRowCells], gm[kRowCells];   // cell's first slot in the sorted arrays, atoms
    int ccell[kRowCells + 1];             // first cell of each class
    float chs[kRowCells][3], clo[kRowCells][3];  // hs and lo of each class
    float red[kRW][32 * kRedRow];         // each warp's home partials at the end of a row
};

// Four neighbour clusters against the row's home cluster: this lane's neighbour atom ja
// (position pj, type tj).  DIAG: the lane's cluster (slot 0) is the home cluster itself
// (pairs with home atom k < jl only); SHIFT: the class adds lo to the difference.
template <int STATS, bool DIAG, bool SHIFT>
__device__ __forceinline__ void row_step(float4 *accum, const float4 *rab, int gs, const float4 &pj,
                                         int tj, int slot, int jl, const f2 (&HX)[4],
                                         const f2 (&HY)[4], const f2 (&HZ)[4], const f2 (&KQ)[4],
                                         f2 (&FX)[4], f2 (&FY)[4], f2 (&FZ)[4], f2 LX, f2 LY,
                                         f2 LZ, float rc2, unsigned &cnt)
{
    const float4 *ab = rab + tj * kRowABStride;
    const f2 X = f2_dup(pj.x), Y = f2_dup(pj.y), Z = f2_dup(pj.z), Q = f2_dup(pj.w);
    const unsigned dm = (DIAG && slot == 0) ? (1u << jl) - 1u : 0xffu;
    f2 RX = 0ull, RY = 0ull, RZ = 0ull;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        f2 dx = f2_sub(HX[p], X), dy = f2_sub(HY[p], Y), dz = f2_sub(HZ[p], Z);
        if (SHIFT) {
            dx = f2_add(dx, LX);
            dy = f2_add(dy, LY);
            dz = f2_add(dz, LZ);
        }
        const f2 r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
        float r2a, r2b;
        f2_split(r2, r2a, r2b);
        bool oka = r2a < rc2, okb = r2b < rc2;
        if (DIAG) {
            oka = oka && ((dm >> (2 * p)) & 1u);
            okb = okb && ((dm >> (2 * p + 1)) & 1u);
        }
        const float4 t = ab[p];  // (A_a, A_b, -B_a, -B_b)
        const f2 A = f2_make(t.x, t.y), nB = f2_make(t.z, t.w);
        const f2 ir = f2_make(rsqrt_hw(r2a), rsqrt_hw(r2b));
        const f2 ir2 = f2_mul(ir, ir);
        const f2 ir6 = f2_mul(f2_mul(ir2, ir2), ir2);
        const f2 kqq = f2_mul(KQ[p], Q);
        // F/r = (kqq / r + (A / r^6 - B) / r^6) / r^2: one product fewer than forming
        // 1/r^8 and kqq / r^2 on their own
        const f2 u = f2_fma(kqq, ir, f2_mul(ir6, f2_fma(A, ir6, nB)));
        float fa, fb;
        f2_split(f2_mul(u, ir2), fa, fb);
        const f2 f = f2_make(oka ? fa : 0.0f, okb ? fb : 0.0f);
        FX[p] = f2_fma(f, dx, FX[p]);
        FY[p] = f2_fma(f, dy, FY[p]);
        FZ[p] = f2_fma(f, dz, FZ[p]);
        RX = f2_fma(f, dx, RX);
        RY = f2_fma(f, dy, RY);
        RZ = f2_fma(f, dz, RZ);
        if (STATS >= kStatsCount) cnt += (unsigned)oka + (unsigned)okb;
    }
    // the reaction on the neighbour atom, added in L2 (a native vector reduction; shared
    // memory has no native float add, and warps of the CTA meet the same atoms)
    float a0, a1, b0, b1, c0, c1;
    f2_split(RX, a0, a1);
    f2_split(RY, b0, b1);
    f2_split(RZ, c0, c1);
    if (gs >= 0) red_add_v4(accum + gs, -(a0 + a1), -(b0 + b1), -(c0 + c1));
}

// The steps of one class list (padded with the dummy cluster to len + 7), each step's
// neighbour atom loaded during the step before.
template <int STATS, bool SHIFT>
__device__ __forceinline__ void row_steps(RowSmem &sm, float4 *accum, const float4 *rab, const unsigned short *lst,
                                          int len, bool diag, int lane, const f2 (&HX)[4],
                                          const f2 (&HY)[4], const f2 (&HZ)[4], const f2 (&KQ)[4],
                                          f2 (&FX)[4], f2 (&FY)[4], f2 (&FZ)[4], f2 LX, f2 LY,
                                          f2 LZ, float rc2, unsigned &cnt)
{
    const int slot = lane >> 3, jl = lane & 7;
    int ja = (int)lst[slot] * kCS + jl;
    float4 pj = sm.np[ja];
    int tj = sm.nt[ja], gs = sm.ng[ja];
    int c0 = 0;
    if (!SHIFT && diag) {
        const int jn = (int)lst[4 + slot] * kCS + jl;
        const float4 pn = sm.np[jn];
        const int tn = sm.nt[jn], gn = sm.ng[jn];
        row_step<STATS, true, false>(accum, rab, gs, pj, tj, slot, jl, HX, HY, HZ, KQ, FX, FY, FZ, LX, LY, LZ, rc2, cnt);
        pj = pn;
        tj = tn;
        gs = gn;
        c0 = 4;
    }
    for (; c0 < len; c0 += 4) {
        const int jn = (int)lst[c0 + 4 + slot] * kCS + jl;
        const float4 pn = sm.np[jn];
        const int tn = sm.nt[jn], gn = sm.ng[jn];
        row_step<STATS, false, SHIFT>(accum, rab, gs, pj, tj, slot, jl, HX, HY, HZ, KQ, FX, FY, FZ, LX, LY, LZ, rc2, cnt);
        pj = pn;
        tj = tn;
        gs = gn;
    }
}

template <int STATS>
__device__ __forceinline__ void row_run(RowSmem &sm, const float2 *s_ab, float4 *rab, const CluArgs &a,
                                        int ic, int mh, int hb, int lane, int T, float kc,
                                        unsigned &cnt)
{
    unsigned short *lst = sm.lst[threadIdx.x >> 5];
    // this row's LJ table: for each neighbour type, (A, A, -B, -B) of home atom pairs
    for (int i = lane; i < T * 4; i += 32) {
        const int tj = i >> 2, p = i & 3;
        const float2 u = s_ab[sm.ht[ic * kCS + 2 * p] * T + tj];
        const float2 v = s_ab[sm.ht[ic * kCS + 2 * p + 1] * T + tj];
        rab[tj * kRowABStride + p] = make_float4(u.x, v.x, u.y, v.y);
    }
    const float4 *hp = sm.hp + ic * kCS;
    f2 KQ[4], FX[4], FY[4], FZ[4], HX[4], HY[4], HZ[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        KQ[p] = f2_make(kc * hp[2 * p].w, kc * hp[2 * p + 1].w);
        FX[p] = FY[p] = FZ[p] = 0ull;
    }
    const float4 bl = sm.hlo[ic], bh = sm.hhi[ic];
    __syncwarp();
    for (int c = 0; c < sm.nclass; ++c) {
        // home coordinates with this class's hs subtracted (exact)
        const float hx = sm.chs[c][0], hy = sm.chs[c][1], hz = sm.chs[c][2];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const float4 u = hp[2 * p], v = hp[2 * p + 1];
            HX[p] = f2_make(u.x - hx, v.x - hx);
            HY[p] = f2_make(u.y - hy, v.y - hy);
            HZ[p] = f2_make(u.z - hz, v.z - hz);
        }
        const float lx = sm.clo[c][0], ly = sm.clo[c][1], lz = sm.clo[c][2];
        const bool shift = lx != 0.0f || ly != 0.0f || lz != 0.0f;
        // the class's clusters in range (the box filter on the shifted home box)
        const float blx = bl.x - hx, bly = bl.y - hy, blz = bl.z - hz;
        const float bhx = bh.x - hx, bhy = bh.y - hy, bhz = bh.z - hz;
        const bool diag = c == 0 && sm.self_nclu > 0;
        const int jb0 = sm.cbeg[sm.ccell[c]], jb1 = sm.cbeg[sm.ccell[c + 1]];
        int len = diag ? 1 : 0;
        if (diag && lane == 0) lst[0] = (unsigned short)ic;
        for (int jb = jb0; jb < jb1; jb += 32) {
            const int jt = jb + lane;
            bool in = false;
            if (jt < jb1 && !(diag && jt <= ic)) {  // the cell itself: clusters after ic
                const float4 nl = sm.nlo[jt], nh = sm.nhi[jt];
                const float gx = fmaxf(0.f, fmaxf(blx - nh.x, nl.x - bhx));
                const float gy = fmaxf(0.f, fmaxf(bly - nh.y, nl.y - bhy));
                const float gz = fmaxf(0.f, fmaxf(blz - nh.z, nl.z - bhz));
                in = gx * gx + gy * gy + gz * gz < a.rc2m;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, in);
            if (in) lst[len + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)jt;
            len += __popc(bal);
        }
        // pad with the dummy cluster: to a multiple of 4, and one step more for the prefetch
        if (lane < 7) lst[len + lane] = (unsigned short)kRowDummy;
        __syncwarp();
        const f2 LX = f2_dup(lx), LY = f2_dup(ly), LZ = f2_dup(lz);
        if (shift)
            row_steps<STATS, true>(sm, static_cast<float4 *>(a.accum), rab, lst, len, diag, lane, HX, HY, HZ, KQ, FX, FY, FZ, LX, LY, LZ, a.rc2, cnt);
        else
            row_steps<STATS, false>(sm, static_cast<float4 *>(a.accum), rab, lst, len, diag, lane, HX, HY, HZ, KQ, FX, FY, FZ, LX, LY, LZ, a.rc2, cnt);
        __syncwarp();
    }
    // the 24 home sums (value 3 k + d: atom k, component d) over the warp: each lane
    // writes its row of partials to the warp's shared array and lane l < 24 sums column l
    float *red = sm.red[threadIdx.x >> 5];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        float a0, a1;
        f2_split(FX[p], a0, a1);
        red[lane * kRedRow + 6 * p + 0] = a0;
        red[lane * kRedRow + 6 * p + 3] = a1;
        f2_split(FY[p], a0, a1);
        red[lane * kRedRow + 6 * p + 1] = a0;
        red[lane * kRedRow + 6 * p + 4] = a1;
        f2_split(FZ[p], a0, a1);
        red[lane * kRedRow + 6 * p + 2] = a0;
        red[lane * kRedRow + 6 * p + 5] = a1;
    }
    __syncwarp();
    if (lane < 24) {
        float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int r = 0; r < 32; r += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] += red[(r + u) * kRedRow + lane];
        }
        const int ia = ic * kCS + lane / 3;
        if (ia < mh)
            atomicAdd(static_cast<float *>(a.accum) + 4 * (size_t)(hb + ia) + lane % 3,
                      (v[0] + v[1]) + (v[2] + v[3]));
    }
    __syncwarp();
}

// One cell of a CTA's group (warp 0 forms and sorts them; the CTA reads them back).
struct RowRec {
    int key, code, beg, cnt, self;  // sort key: the cell itself, then no wrap, then by code
    float hs[3], ns[3], lo[3];
};
constexpr int kHomeIter = kRowCellAtoms / kRT;               // home slots per thread


template <int STATS>
__global__ void __launch_bounds__(kRT, 4)
k_cluster_rows(CluArgs a, int ncells)
{
    __shared__ __align__(16) union RowUnion {
        RowSmem r;
        CluSmem<MD_ACCUM_F32> c;
    } u;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    const int T = a.ntypes;
    float2 *s_ab = reinterpret_cast<float2 *>(s_dyn);  // [T * T]: (A, -B)
    float4 *s_rab = reinterpret_cast<float4 *>(s_dyn + ((sizeof(float2) * T * T + 15) & ~(size_t)15));
    pdl_wait();
    pdl_trigger();
    const int cell = blockIdx.x, grp = blockIdx.y;
    const int hb = a.cell_start[cell], mh = a.cell_start[cell + 1] - hb;
    // the group's cells, sorted into classes of equal wrap code (the cell itself first),
    // formed by warp 0 and shared
    __shared__ RowRec s_rec[kRowCells];
    __shared__ int s_ne;
    RowRec r[kRowCells];
    int ne = 0;
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < kRowCells; ++k) {
            const int e = kRowGroup[grp][k];
            r[k].key = 1 << 20;
            r[k].code = -1;
            r[k].beg = r[k].cnt = r[k].self = 0;
#pragma unroll
            for (int d = 0; d < 3; ++d) r[k].hs[d] = r[k].ns[d] = r[k].lo[d] = 0.0f;
            if (e >= 0) {
                PairGeom q;
                const int code = forward_pair(a.box, cell, e, q);
                r[k].code = code;
                r[k].self = q.self;
                r[k].key = q.self ? -2 : (code == 13 ? -1 : code);
                r[k].beg = a.cell_start[q.nbr];
                r[k].cnt = a.cell_start[q.nbr + 1] - r[k].beg;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    r[k].hs[d] = q.hs[d];
                    r[k].ns[d] = q.ns[d];
                    r[k].lo[d] = q.lo[d];
                }
                ++ne;
            }
        }
#pragma unroll
        for (int i = 0; i < kRowCells - 1; ++i) {
#pragma unroll
            for (int j = 0; j < kRowCells - 1 - i; ++j) {
                if (r[j].key > r[j + 1].key) {
                    const RowRec t = r[j];
                    r[j] = r[j + 1];
                    r[j + 1] = t;
                }
            }
        }
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < kRowCells; ++k) s_rec[k] = r[k];
            s_ne = ne;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRowCells; ++k) r[k] = s_rec[k];
    ne = s_ne;
    bool fits = mh <= kRowCellAtoms;
#pragma unroll
    for (int k = 0; k < kRowCells; ++k) fits = fits && r[k].cnt <= kRowCellAtoms;
    if (!fits) {
        for (int k = 0; k < ne; ++k)
            cluster_item<MD_ACCUM_F32, STATS, false, false>(u.c, s_ab, a, BatchArgs{}, nullptr, cell,
                                                           kEntrySlot[kRowGroup[grp][k]], ncells);
        return;
    }
    RowSmem &sm = u.r;
    int cb[kRowCells + 1];
    cb[0] = 0;
#pragma unroll
    for (int k = 0; k < kRowCells; ++k) cb[k + 1] = cb[k] + (r[k].cnt + kCS - 1) / kCS;
    const int ncl = cb[kRowCells];
    if (threadIdx.x == 0) {
        int ncls = 0;
#pragma unroll
        for (int k = 0; k < kRowCells; ++k) {
            if (k < ne && (k == 0 || r[k].code != r[k - 1].code)) {
                sm.ccell[ncls] = k;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    sm.chs[ncls][d] = r[k].hs[d];
                    sm.clo[ncls][d] = r[k].lo[d];
                }
                ++ncls;
            }
            sm.gbeg[k] = r[k].beg;
            sm.gm[k] = r[k].cnt;
            sm.cbeg[k] = cb[k];
        }
        sm.cbeg[kRowCells] = ncl;
        sm.ccell[ncls] = ne;
        sm.nclass = ncls;
        sm.ncl = ncl;
        sm.self_nclu = r[0].self ? (mh + kCS - 1) / kCS : 0;
        sm.next = kRW;
    }
    for (int t = threadIdx.x; t < T * T; t += kRT) {
        const float2 ab = a.AB[t];
        s_ab[t] = make_float2(ab.x, -ab.y);
    }
    // every load of a thread (home and neighbour tiles, cluster boxes) issued before its
    // stores: at most 256 atoms (32 clusters) per cell, so two slots of each cell and one
    // cluster of each cell per thread
    float4 hv[kHomeIter];
    int hty[kHomeIter];
#pragma unroll
    for (int i = 0; i < kHomeIter; ++i) {
        const int t = threadIdx.x + i * kRT;
        if (t < mh) {
            hv[i] = a.pq[hb + t];
            hty[i] = a.ty[hb + t];
        }
    }
    const int nic = (mh + kCS - 1) / kCS;
    float4 hbl, hbh;
    if (threadIdx.x < nic) {
        hbl = a.cbox[hb + threadIdx.x * kCS];
        hbh = a.cbox[(size_t)a.n + hb + threadIdx.x * kCS];
    }
    float4 v[kRowCells][2], bl[kRowCells], bh[kRowCells];
    int ty[kRowCells][2];
#pragma unroll
    for (int k = 0; k < kRowCells; ++k) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int t = threadIdx.x + i * kRT;
            if (t < r[k].cnt) {
                v[k][i] = a.pq[r[k].beg + t];
                ty[k][i] = a.ty[r[k].beg + t];
            }
        }
        if (threadIdx.x * kCS < r[k].cnt) {
            bl[k] = a.cbox[r[k].beg + threadIdx.x * kCS];
            bh[k] = a.cbox[(size_t)a.n + r[k].beg + threadIdx.x * kCS];
        }
    }
    // home tile (as stored) and types, padding at +far; home cluster boxes
#pragma unroll
    for (int i = 0; i < kHomeIter; ++i) {
        const int t = threadIdx.x + i * kRT;
        if (t < nic * kCS) {
            const bool hr = t < mh;
            sm.hp[t] = hr ? hv[i] : make_float4(kFar, kFar, kFar, 0.f);
            sm.ht[t] = (unsigned char)(hr ? clamp_type(hty[i], T, a.status) : 0);
        }
    }
    if (threadIdx.x < nic) {
        sm.hlo[threadIdx.x] = hbl;
        sm.hhi[threadIdx.x] = hbh;
    }
    // neighbour tiles in class order, ns subtracted (exact), padding at -far; their boxes
    // moved by the same shift
#pragma unroll
    for (int k = 0; k < kRowCells; ++k) {
        const int s0 = cb[k] * kCS, span = (cb[k + 1] - cb[k]) * kCS;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int t = threadIdx.x + i * kRT;
            if (t < span) {
                float4 p = make_float4(-kFar, -kFar, -kFar, 0.f);
                int tt = 0;
                if (t < r[k].cnt) {
                    p = v[k][i];
                    p.x -= r[k].ns[0];
                    p.y -= r[k].ns[1];
                    p.z -= r[k].ns[2];
                    tt = clamp_type(ty[k][i], T, a.status);
                }
                sm.np[s0 + t] = p;
                sm.nt[s0 + t] = (unsigned char)tt;
                sm.ng[s0 + t] = t < r[k].cnt ? r[k].beg + t : -1;
            }
        }
        if (threadIdx.x * kCS < r[k].cnt) {
            const int c = cb[k] + threadIdx.x;
            sm.nlo[c] = make_float4(bl[k].x - r[k].ns[0], bl[k].y - r[k].ns[1], bl[k].z - r[k].ns[2], 0.f);
            sm.nhi[c] = make_float4(bh[k].x - r[k].ns[0], bh[k].y - r[k].ns[1], bh[k].z - r[k].ns[2], 0.f);
        }
    }
    if (threadIdx.x < kCS) {
        const int s = kRowDummy * kCS + threadIdx.x;
        sm.np[s] = make_float4(-kFar, -kFar, -kFar, 0.f);
        sm.nt[s] = 0;
        sm.ng[s] = -1;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *rab = s_rab + (size_t)warp * T * kRowABStride;
    unsigned cnt = 0;
    for (int ic = warp; ic < nic;) {
        row_run<STATS>(sm, s_ab, rab, a, ic, mh, hb, lane, T, a.kc, cnt);
        int nx = 0;
        if (lane == 0) nx = atomicAdd(&sm.next, 1);
        ic = __shfl_sync(0xffffffffu, nx, 0);
    }
    if (STATS != kStatsNone) {
        // the group's count in the partial of its first entry, zero in the others
        Partial *partials = a.partials;
        block_partial_to<kRT>(0.0, 0.0, 0.0, (unsigned long long)cnt,
                              partials + (size_t)kEntrySlot[kRowGroup[grp][0]] * ncells + cell);
        if (threadIdx.x == 0)
            for (int k = 1; k < ne; ++k)
                partials[(size_t)kEntrySlot[kRowGroup[grp][k]] * ncells + cell] = Partial{0.0, 0.0, 0.0, 0ull};
    }
}

// Cluster-order accumulators -> forces_out in input order (slot s holds the atom
// perm[corder[s]], or perm[s] without corder).  KICK: the half kick v += dt/2 a(F) of
// that atom in the same pass, with the arithmetic of k_kick.
template <int MODE, bool KICK>
__global__ void __launch_bounds__(256)
k_finalize_clu(const void *__restrict__ accum, const int32_t *__restrict__ corder,
               const int32_t *__restrict__ perm, int n, void *__restrict__ forces_out,
               uint32_t *status, double *__restrict__ vel, const float *__restrict__ inv_mass,
               double half_dt)
{
    pdl_wait();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int o = perm[corder ? corder[s] : s];
    double f[3];
    if (MODE == MD_ACCUM_FIXED64) {
        const long long *acc = static_cast<const long long *>(accum);
        long long *F = static_cast<long long *>(forces_out);
        const long long v[3] = {acc[s], acc[(size_t)n + s], acc[2 * (size_t)n + s]};
        const double sc = 1.0 / 4294967296.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            F[3 * o + k] = v[k];
            f[k] = (double)v[k] * sc;
        }
    } else {
        const float4 v = static_cast<const float4 *>(accum)[s];
        float *F = static_cast<float *>(forces_out);
        F[3 * o + 0] = v.x;
        F[3 * o + 1] = v.y;
        F[3 * o + 2] = v.z;
        if (!isfinite(v.x + v.y + v.z)) set_status(status, MD_STATUS_NONFINITE);
        f[0] = v.x;
        f[1] = v.y;
        f[2] = v.z;
    }
    if (KICK) {
        const double c = kick_factor((double)inv_mass[o], half_dt);
#pragma unroll
        for (int k = 0; k < 3; ++k) vel[3 * o + k] = kick_velocity(vel[3 * o + k], f[k], c);
    }
}

// grid: cells x stencil entries x shares of a cell pair (kMiSplit for boxes with an axis
// of 2 cells, else 1).  PERSIST: the same items from about one wave of CTAs (blocks per
// SM at this launch's shared memory x SMs), taking items from `work`.
template <int MODE, int STATS, bool BATCHED = false, bool MI = false, bool PERSIST = false,
          bool GATHER = false>
cudaError_t launch_cluster_t(const CluArgs &c, dim3 grid, cudaStream_t stream,
                             const BatchArgs &b = BatchArgs{},
                             unsigned long long *sys_pair_count = nullptr, int *work = nullptr)
{
    const size_t dyn = sizeof(float2) * (size_t)c.ntypes * (size_t)c.ntypes;
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_cluster<MODE, STATS, BATCHED, MI, PERSIST, GATHER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)(sizeof(float2) * kMaxTypes * kMaxTypes));
    (void)attr;
    dim3 g = grid;
    if (PERSIST) {
        // one wave at this launch's shared memory (host queries only; no stream work)
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cluster<MODE, STATS, BATCHED, MI, PERSIST, GATHER>,
                                                      kCT, dyn);
        const long long wave = (long long)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
        const long long items = (long long)grid.x * grid.y * grid.z;
        g = dim3((unsigned)(items < wave ? items : wave), 1);
    }
    return launch_pdl(k_cluster<MODE, STATS, BATCHED, MI, PERSIST, GATHER>, g, dim3(kCT), dyn, stream, c, b,
                      sys_pair_count, work, (int)grid.x, (int)grid.y, (int)grid.z);
}

template <int MODE, bool MI, bool GATHER = false>
cudaError_t launch_cluster_stats(int stats, const CluArgs &c, dim3 grid, cudaStream_t stream)
{
    if (stats == kStatsEnergy) return launch_cluster_t<MODE, kStatsEnergy, false, MI, false, GATHER>(c, grid, stream);
    // the Verlet step asks for forces, or forces and energies
    if (stats == kStatsCount && !GATHER) return launch_cluster_t<MODE, kStatsCount, false, MI>(c, grid, stream);
    return launch_cluster_t<MODE, kStatsNone, false, MI, false, GATHER>(c, grid, stream);
}

// SMs of the current device (host query, cached per device).
int device_sms()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!cached[dev]) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = sms > 0 ? sms : 1;
    }
    return cached[dev];
}

// The long-row form: grid (cells, groups); partials in the one-cluster-pair grid's layout.
cudaError_t launch_cluster_rows(int stats, const CluArgs &c, int ncells, cudaStream_t stream)
{
    const size_t dyn = ((sizeof(float2) * (size_t)c.ntypes * c.ntypes + 15) & ~(size_t)15) +
                       sizeof(float4) * kRW * (size_t)c.ntypes * kRowABStride;
    const size_t dyn_max = sizeof(float2) * kMaxTypes * kMaxTypes + sizeof(float4) * kRW * kMaxTypes * kRowABStride;
    const dim3 grid(ncells, kRowGroups);
    if (stats == kStatsCount) {
        static const cudaError_t attr = cudaFuncSetAttribute(
            k_cluster_rows<kStatsCount>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
        (void)attr;
        return launch_pdl(k_cluster_rows<kStatsCount>, grid, dim3(kRT), dyn, stream, c, ncells);
    }
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_cluster_rows<kStatsNone>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
    (void)attr;
    return launch_pdl(k_cluster_rows<kStatsNone>, grid, dim3(kRT), dyn, stream, c, ncells);
}

template <int MODE>
cudaError_t launch_cluster_mode(bool mi, bool gather, int stats, const CluArgs &c, dim3 grid,
                                cudaStream_t stream)
{
    if (gather)
        return mi ? launch_cluster_stats<MODE, true, true>(stats, c, grid, stream)
                  : launch_cluster_stats<MODE, false, true>(stats, c, grid, stream);
    return mi ? launch_cluster_stats<MODE, true>(stats, c, grid, stream)
              : launch_cluster_stats<MODE, false>(stats, c, grid, stream);
}

}  // namespace

cudaError_t launch_cluster(const ForceArgs &a, const WsLayout &ws, char *wsp, Partial *partials,
                           int *nblocks_out, cudaStream_t stream)
{
    const size_t acc_bytes = (size_t)a.n * (fixed_output(a.mode) ? 24 : 16);
    void *accum = wsp + ws.accum;
    float4 *cpq = reinterpret_cast<float4 *>(wsp + ws.clu_pos_q);
    int32_t *cty = reinterpret_cast<int32_t *>(wsp + ws.clu_type);
    int32_t *corder = reinterpret_cast<int32_t *>(wsp + ws.clu_order);
    float4 *cbox = reinterpret_cast<float4 *>(wsp + ws.clu_box);
    // the MD step's build pass, or else the ordering pass, zeroes the accumulators; a
    // presorted call without that needs the memset
    cudaError_t e = a.accum_zeroed || !a.presorted ? cudaSuccess : cudaMemsetAsync(accum, 0, acc_bytes, stream);
    if (e != cudaSuccess) return e;
    if (!a.presorted)
        k_cluster_order<<<a.box.ncell, kOrderThreads, 0, stream>>>(a.cell_start, a.pos_q_sorted,
                                                                   a.type_sorted, a.box, cpq, cty, corder,
                                                                   accum, a.mode, a.n, cbox);
    CluArgs c;
    c.cell_start = a.cell_start;
    c.pq = a.presorted ? a.pos_q_sorted : cpq;
    c.ty = a.presorted ? a.type_sorted : cty;
    c.box = a.box;
    c.AB = a.AB;
    c.ntypes = a.ntypes;
    c.kc = a.k_coulomb;
    const int per_cell = half_shell_pairs_per_cell(a.box);
    const bool mi = per_cell == 27;  // an axis of 2 cells: per-pair minimum image
    cutoff_thresholds(a.box, a.rc64, mi, &c.rc2, &c.rc2m);
    c.accum = accum;
    c.n = a.n;
    c.partials = partials;
    c.status = a.status;
    c.gpq = a.gather_pq;
    c.perm = a.perm;
    c.cbox = a.presorted ? a.clu_box : cbox;
    const bool gather = a.gather_pq != nullptr;
    if (gather && !a.presorted) return cudaErrorInvalidValue;
    // a system alone with an axis of 2 cells: its few long cell pairs split over kMiSplit
    // CTAs (not in MD_ACCUM_FIXED_TILE, whose rounding points would move, and whose single
    // and batched results are the same bits; batches fill the GPU without it)
    dim3 grid(a.box.ncell, per_cell, mi && a.mode != MD_ACCUM_FIXED_TILE ? kMiSplit : 1);
    const int stats = a.energy_virial_out ? kStatsEnergy : (a.pair_count_out ? kStatsCount : kStatsNone);
    // the long-row form where its grid (4 CTAs a cell) fills at least one wave of 4 CTAs
    // per SM and the cells hold at most 225 atoms on average (fuller cells more often
    // exceed its 256-atom tiles); elsewhere the one-cluster-pair grid (14 CTAs a cell) was
    // measured faster
    if (a.mode == MD_ACCUM_F32 && !mi && !gather && stats != kStatsEnergy && c.cbox &&
        (long long)a.box.ncell * kRowGroups >= 4LL * device_sms() &&
        (long long)a.n <= 225LL * a.box.ncell)
        e = launch_cluster_rows(stats, c, a.box.ncell, stream);
    else if (a.mode == MD_ACCUM_FIXED64)
        e = launch_cluster_mode<MD_ACCUM_FIXED64>(mi, gather, stats, c, grid, stream);
    else if (a.mode == MD_ACCUM_FIXED_TILE)
        e = launch_cluster_mode<MD_ACCUM_FIXED_TILE>(mi, gather, stats, c, grid, stream);
    else
        e = launch_cluster_mode<MD_ACCUM_F32>(mi, gather, stats, c, grid, stream);
    *nblocks_out = a.box.ncell * per_cell * (int)grid.z;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_finalize_cluster(a, accum, ws, wsp, a.n, stream);
}

template <int MODE, bool MI, bool PERSIST>
cudaError_t launch_cluster_batched_t(const CluArgs &c, dim3 grid, cudaStream_t stream, const BatchArgs &b,
                              unsigned long long *cnt, int *work)
{
    if (cnt) return launch_cluster_t<MODE, kStatsCount, true, MI, PERSIST>(c, grid, stream, b, cnt, work);
    return launch_cluster_t<MODE, kStatsNone, true, MI, PERSIST>(c, grid, stream, b, nullptr, work);
}

// Batched cluster kernel over the regular systems' cells (b.cell_list[0 .. ncell_reg),
// 14 cell pairs each) or, mi, over those of the systems with a 2-cell axis (27 each).
// persist_work: the persistent grid with this zeroed counter, else one CTA per pair.
cudaError_t launch_cluster_batched(int mode, bool mi, const BatchArgs &b, const int32_t *cell_start,
                                   const float4 *pq, const int32_t *ty, void *accum,
                                   Partial *partials, uint32_t *status,
                                   unsigned long long *sys_pair_count, int *persist_work,
                                   cudaStream_t stream)
{
    const int ncells = mi ? b.ncell_mi : b.ncell_reg;
    if (ncells <= 0) return cudaSuccess;
    CluArgs c = {};
    c.cell_start = cell_start;
    c.pq = pq;  // cluster-ordered tiles
    c.ty = ty;
    c.ntypes = b.max_ntypes;  // sizes the shared LJ table
    c.accum = accum;
    c.n = b.n;
    c.partials = partials;
    c.status = status;
    dim3 grid(ncells, mi ? 27 : 14);
    unsigned long long *cnt = sys_pair_count;
    int *w = persist_work;
    const int sel = (mode == MD_ACCUM_FIXED64 ? 4 : mode == MD_ACCUM_FIXED_TILE ? 8 : 0) + (mi ? 2 : 0) + (w ? 1 : 0);
    cudaError_t e;
    switch (sel) {
    case 0: e = launch_cluster_batched_t<MD_ACCUM_F32, false, false>(c, grid, stream, b, cnt, w); break;
    case 1: e = launch_cluster_batched_t<MD_ACCUM_F32, false, true>(c, grid, stream, b, cnt, w); break;
    case 2: e = launch_cluster_batched_t<MD_ACCUM_F32, true, false>(c, grid, stream, b, cnt, w); break;
    case 3: e = launch_cluster_batched_t<MD_ACCUM_F32, true, true>(c, grid, stream, b, cnt, w); break;
    case 4: e = launch_cluster_batched_t<MD_ACCUM_FIXED64, false, false>(c, grid, stream, b, cnt, w); break;
    case 5: e = launch_cluster_batched_t<MD_ACCUM_FIXED64, false, true>(c, grid, stream, b, cnt, w); break;
    case 6: e = launch_cluster_batched_t<MD_ACCUM_FIXED64, true, false>(c, grid, stream, b, cnt, w); break;
    case 7: e = launch_cluster_batched_t<MD_ACCUM_FIXED64, true, true>(c, grid, stream, b, cnt, w); break;
    case 8: e = launch_cluster_batched_t<MD_ACCUM_FIXED_TILE, false, false>(c, grid, stream, b, cnt, w); break;
    case 9: e = launch_cluster_batched_t<MD_ACCUM_FIXED_TILE, false, true>(c, grid, stream, b, cnt, w); break;
    case 10: e = launch_cluster_batched_t<MD_ACCUM_FIXED_TILE, true, false>(c, grid, stream, b, cnt, w); break;
    default: e = launch_cluster_batched_t<MD_ACCUM_FIXED_TILE, true, true>(c, grid, stream, b, cnt, w); break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Cluster-order accumulators -> forces in input order (batched or not), with the half
// kick when a.kick_vel is set.
cudaError_t launch_finalize_cluster(const ForceArgs &a, const void *accum, const WsLayout &ws,
                                    char *wsp, int n, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    const int32_t *corder = a.presorted ? nullptr : reinterpret_cast<const int32_t *>(wsp + ws.clu_order);
    const int g = (n + 255) / 256;
    const bool kick = a.kick_vel != nullptr;
    const dim3 blk(256);
    cudaError_t e;
    if (fixed_output(a.mode)) {  // int64 accumulators (FIXED64 and FIXED_TILE alike)
        if (kick)
            e = launch_pdl(k_finalize_clu<MD_ACCUM_FIXED64, true>, dim3(g), blk, 0, stream, accum, corder, a.perm, n, a.forces_out, a.status, a.kick_vel, a.kick_inv_mass, a.kick_half_dt);
        else
            e = launch_pdl(k_finalize_clu<MD_ACCUM_FIXED64, false>, dim3(g), blk, 0, stream, accum, corder, a.perm, n, a.forces_out, a.status, (double *)nullptr, (const float *)nullptr, 0.0);
    } else {
        if (kick)
            e = launch_pdl(k_finalize_clu<MD_ACCUM_F32, true>, dim3(g), blk, 0, stream, accum, corder, a.perm, n, a.forces_out, a.status, a.kick_vel, a.kick_inv_mass, a.kick_half_dt);
        else
            e = launch_pdl(k_finalize_clu<MD_ACCUM_F32, false>, dim3(g), blk, 0, stream, accum, corder, a.perm, n, a.forces_out, a.status, (double *)nullptr, (const float *)nullptr, 0.0);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace mdnb
