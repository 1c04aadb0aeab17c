// md_forces_half.cu -- half-shell cell-pair force kernel (MD_ALGO_HALF_SHELL).
//
// The loop nest of Algorithm 1 with every unordered pair met once: each CTA takes one
// (home cell, neighbour cell) pair of the half shell (the home cell itself with i<j,
// plus 13 forward neighbours), and the reaction -F goes to the neighbour atom
// (Newton's third law).  The two stages of the paper's enhanced accelerator
// (Section V.B: cheap distance filters feeding one expensive force unit through a
// FIFO) become, inside one warp and one 32x32 item (32 home rows x 32 neighbour
// columns):
//   filter:  each lane holds one home atom; the 32 neighbour atoms are broadcast from
//            shared memory; the sign of rc'^2 - r^2 of every candidate is folded into
//            a 32-bit row mask with one funnel shift;
//   compact: a popcount prefix sum over the rows gives each row its offset, and the
//            surviving (row, column) pairs are written contiguously per row;
//   force:   full warps of 32 survivors evaluate Eq. 1 + Eq. 2, so a low survival rate
//            does not idle lanes of the force math.  The exact test r^2 < rc^2 is
//            applied here; the filter uses rc'^2 = rc^2 + a tiny margin so that it
//            never rejects a pair the exact test keeps;
//   reduce:  each lane sums its own row's contiguous pair forces into registers (the
//            i-side, kept across the whole row block); the survival matrix is
//            transposed with warp shuffles so that each lane gathers its column's
//            pair forces (the j-side reaction) into warp-private shared arrays.
// No atomics are used until a tile is finished; then one vector atomic per atom.
//
// Periodic images and cell pairs: md_pairgeom.cuh.
#include <math.h>

#include "md_internal.cuh"
#include "md_pairgeom.cuh"

namespace mdnb {
namespace {

constexpr int kHWDefault = 4;        // warps per CTA of the single-system launches
constexpr int kTile = 256;           // atoms of a cell staged at once (i, j indices fit 8 bits)

struct HalfArgs {
    const int32_t *cell_start;
    const float4 *pq;
    const int32_t *ty;
    BoxF box;
    const float2 *AB;
    int ntypes;
    float kc;
    float rc2;   // exact cutoff test
    float rc2m;  // filter threshold (conservative)
    void *accum; // float4[n] (F32) or u64[3][n] (FIXED64), sorted order, zeroed
    int n;
    Partial *partials;
    uint32_t *status;
};

// 32x32 bit-matrix transpose across a warp: lane l holds row l (bit k = M[l][k]) on
// entry and column l (bit k = M[k][l]) on exit.
__device__ __forceinline__ unsigned transpose32(unsigned x, int lane)
{
    const unsigned lo[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const int s = 16 >> t;
        const unsigned y = __shfl_xor_sync(0xffffffffu, x, s);
        x = (lane & s) ? ((x & ~lo[t]) | ((y & ~lo[t]) >> s)) : ((x & lo[t]) | ((y & lo[t]) << s));
    }
    return x;
}

// Bounding box of each 32-atom block of a staged tile (padding slots excluded), one
// warp per block.  Blocks with no atom get an empty box that is never in range.
template <int W>
__device__ __forceinline__ void block_boxes(const float (*xyz)[kTile], int m, int m32,
                                            float (*box)[6])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = warp; b < (m32 >> 5); b += W) {
        const int t = b * 32 + lane;
        const bool in = t < m;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float lo = in ? xyz[d][t] : kFar, hi = in ? xyz[d][t] : -kFar;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            if (lane == 0) {
                box[b][d] = lo;
                box[b][d + 3] = hi;
            }
        }
    }
    __syncthreads();
}

template <int MODE>
struct KCap {
    // survivors buffered per pass (default): one pass holds a typical 32x32 item
    static constexpr int value = MODE == MD_ACCUM_FIXED64 ? 128 : 256;
};

template <int MODE>
__device__ __forceinline__ void smem_add(typename AccT<MODE>::T *p, typename AccT<MODE>::T v)
{
    if (MODE == MD_ACCUM_FIXED64)
        atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
    else
        atomicAdd(reinterpret_cast<float *>(p), (float)v);
}

// W warps per CTA and CAP buffered survivors per warp are the tunable shape; the launch
// bound keeps 64 registers per thread for every W.
template <int MODE, bool ENERGY, bool MI, bool BATCHED, int W, int CAP>
__global__ void __launch_bounds__(W * 32, 32 / W)
k_half_shell(HalfArgs a, BatchArgs b, unsigned long long *sys_pair_count)
{
    using Acc = typename AccT<MODE>::T;
    constexpr int kHW = W;
    constexpr int kHT = W * 32;
    __shared__ __align__(16) float s_hxyz[3][kTile];  // home tile (box shift applied)
    __shared__ __align__(16) float s_nxyz[3][kTile];  // neighbour tile
    __shared__ float s_hq[kTile], s_nq[kTile];
    __shared__ int s_ht[kTile], s_nt[kTile];
    __shared__ float s_hbox[kTile / 32][6];  // per 32-atom block: lo xyz, hi xyz
    __shared__ float s_nbox[kTile / 32][6];
    __shared__ Acc s_hf[3][kTile];           // forces on home atoms (whole cell pair)
    __shared__ Acc s_nf[3][kTile];           // reactions on neighbour atoms (this tile)
    __shared__ uint16_t s_q[kHW][CAP];       // per-warp (row, column) of buffered pairs
    __shared__ uint16_t s_cl[kHW][CAP];      // the same pairs in column order: buffer index
    __shared__ unsigned s_col[kHW][32];      // per-warp column masks (rows keeping column k)
    __shared__ int s_cs[kHW][32];            // per-warp column offsets within the pass
    // dynamic: per-warp pair forces of the current item pass [kHW][3][CAP], then the LJ
    // table [ntypes * ntypes]
    extern __shared__ __align__(16) unsigned char s_dyn[];
    Acc(*s_fb)[3][CAP] = reinterpret_cast<Acc(*)[3][CAP]>(s_dyn);
    float2 *s_ab = reinterpret_cast<float2 *>(s_dyn + sizeof(Acc) * kHW * 3 * CAP);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float e_lj = 0.f, e_c = 0.f, vir = 0.f;
    unsigned long long cnt = 0;

    // the system this CTA works on: the only one, or the one its cell belongs to
    PairGeom g;
    bool valid;
    int T, sid = 0;
    const float2 *AB;
    float kc, rc2, rc2m;
    MiBox mb;
    if (BATCHED) {
        const int cell = b.cell_list[(MI ? b.ncell_reg : 0) + blockIdx.x];
        sid = b.cell_sys[cell];
        const SysDesc &d = b.sys[sid];
        valid = cell_pair(d.box, cell - d.cell_offset, blockIdx.y, g);
        g.home += d.cell_offset;
        g.nbr += d.cell_offset;
        T = d.ntypes;
        AB = d.AB;
        kc = d.kc;
        rc2 = d.rc2;
        rc2m = d.rc2m;
        if (MI)
            for (int k = 0; k < 3; ++k) { mb.Lhi[k] = d.box.Lhi[k]; mb.Llo[k] = d.box.Llo[k]; mb.invL[k] = d.box.invL[k]; }
    } else {
        valid = cell_pair(a.box, blockIdx.x, blockIdx.y, g);
        T = a.ntypes;
        AB = a.AB;
        kc = a.kc;
        rc2 = a.rc2;
        rc2m = a.rc2m;
        if (MI)
            for (int k = 0; k < 3; ++k) { mb.Lhi[k] = a.box.Lhi[k]; mb.Llo[k] = a.box.Llo[k]; mb.invL[k] = a.box.invL[k]; }
    }
    if (!valid) {
        block_partial<kHT>(0.0, 0.0, 0.0, 0ull, a.partials + (size_t)blockIdx.y * gridDim.x);
        return;
    }
    const int h_begin = a.cell_start[g.home], nh = a.cell_start[g.home + 1] - h_begin;
    const int n_begin = a.cell_start[g.nbr], nn = a.cell_start[g.nbr + 1] - n_begin;
    if (nh == 0 || nn == 0) {
        block_partial<kHT>(0.0, 0.0, 0.0, 0ull, a.partials + (size_t)blockIdx.y * gridDim.x);
        return;
    }
    for (int t = threadIdx.x; t < T * T; t += kHT) s_ab[t] = AB[t];
    uint16_t *q = s_q[warp];
    Acc(*fb)[CAP] = s_fb[warp];

    for (int h0 = 0; h0 < nh; h0 += kTile) {
        const int mh = min(kTile, nh - h0);
        const int mh32 = (mh + 31) & ~31;
        __syncthreads();
        for (int t = threadIdx.x; t < mh32; t += kHT) {
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
            s_hxyz[0][t] = p.x;
            s_hxyz[1][t] = p.y;
            s_hxyz[2][t] = p.z;
            s_hq[t] = p.w;
            s_ht[t] = ty;
            s_hf[0][t] = s_hf[1][t] = s_hf[2][t] = Acc(0);
        }
        __syncthreads();
        block_boxes<W>(s_hxyz, mh, mh32, s_hbox);
        for (int n0 = g.self ? h0 : 0; n0 < nn; n0 += kTile) {
            const int mn = min(kTile, nn - n0);
            const bool diag = g.self && n0 == h0;
            const int mn32 = (mn + 31) & ~31;
            // neighbour tile (for the home cell's own tile: a copy of the home tile, so
            // that every access below names a fixed shared array)
            __syncthreads();
            for (int t = threadIdx.x; t < mn32; t += kHT) {
                if (diag) {
                    s_nxyz[0][t] = s_hxyz[0][t];
                    s_nxyz[1][t] = s_hxyz[1][t];
                    s_nxyz[2][t] = s_hxyz[2][t];
                    s_nq[t] = s_hq[t];
                    s_nt[t] = s_ht[t];
                } else {
                    float4 p;
                    int ty = 0;
                    if (t < mn) {
                        p = a.pq[n_begin + n0 + t];
                        p.x -= g.ns[0];
                        p.y -= g.ns[1];
                        p.z -= g.ns[2];
                        ty = clamp_type(a.ty[n_begin + n0 + t], T, a.status);
                    } else {
                        p = make_float4(-kFar, -kFar, -kFar, 0.f);
                    }
                    s_nxyz[0][t] = p.x;
                    s_nxyz[1][t] = p.y;
                    s_nxyz[2][t] = p.z;
                    s_nq[t] = p.w;
                    s_nt[t] = ty;
                }
                s_nf[0][t] = s_nf[1][t] = s_nf[2][t] = Acc(0);
            }
            __syncthreads();
            if (diag) {
                for (int t = threadIdx.x; t < (mn32 >> 5) * 6; t += kHT) s_nbox[t / 6][t % 6] = s_hbox[t / 6][t % 6];
                __syncthreads();
            } else {
                block_boxes<W>(s_nxyz, mn, mn32, s_nbox);
            }

            const int nib = mh32 >> 5, njb = mn32 >> 5;
            const int nitems = diag ? nib * (nib + 1) / 2 : nib * njb;
            int cur_ib = -1;
            Acc ax = Acc(0), ay = Acc(0), az = Acc(0);  // i-side sums while the row block stays
            float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
            unsigned long long xi2 = 0ull, yi2 = 0ull, zi2 = 0ull;
            const unsigned long long nrc2 = f2_dup(-rc2m);
            for (int it = warp; it < nitems; it += kHW) {
                int ib, jb;
                if (diag) {
                    int r = it;
                    ib = 0;
                    while (r >= nib - ib) { r -= nib - ib; ++ib; }
                    jb = ib + r;
                } else {
                    ib = it / njb;
                    jb = it - ib * njb;
                }
                const int i = ib * 32 + lane;
                if (ib != cur_ib) {
                    if (cur_ib >= 0 && cur_ib * 32 + lane < mh) {
                        const int ii = cur_ib * 32 + lane;
                        smem_add<MODE>(&s_hf[0][ii], ax);
                        smem_add<MODE>(&s_hf[1][ii], ay);
                        smem_add<MODE>(&s_hf[2][ii], az);
                    }
                    ax = ay = az = Acc(0);
                    cur_ib = ib;
                    pi = make_float4(s_hxyz[0][i], s_hxyz[1][i], s_hxyz[2][i], s_hq[i]);
                    xi2 = f2_dup(pi.x);
                    yi2 = f2_dup(pi.y);
                    zi2 = f2_dup(pi.z);
                }
                if (!MI) {
                    // the whole item is out of range if the two blocks' boxes are rc'
                    // apart (every pair in it would fail the filter)
                    const float *hb = s_hbox[ib], *nb = s_nbox[jb];
                    const float gx = fmaxf(0.f, fmaxf(hb[0] - nb[3], nb[0] - hb[3]));
                    const float gy = fmaxf(0.f, fmaxf(hb[1] - nb[4], nb[1] - hb[4]));
                    const float gz = fmaxf(0.f, fmaxf(hb[2] - nb[5], nb[2] - hb[5]));
                    if (gx * gx + gy * gy + gz * gz >= rc2m) continue;
                }
                // ---- filter: bit jj of keep <-> neighbour slot jb*32 + jj
                unsigned keep;
                if (MI) {
                    unsigned fail = 0u;
#pragma unroll 8
                    for (int jj = 31; jj >= 0; --jj) {
                        const int jt = jb * 32 + jj;
                        const float4 pj = make_float4(s_nxyz[0][jt], s_nxyz[1][jt], s_nxyz[2][jt], 0.f);
                        float dx, dy, dz;
                        displacement<true>(pi, pj, g, mb, dx, dy, dz);
                        const float s = fmaf(-dz, dz, fmaf(-dy, dy, fmaf(-dx, dx, rc2m)));
                        // (fail << 1) | sign(s): a negative s rejects the candidate
                        fail = __funnelshift_l(__float_as_uint(s), fail, 1);
                    }
                    keep = ~fail;
                } else {
                    // two candidates per packed instruction; s = r^2 - rc'^2 is negative
                    // exactly for the candidates to keep
                    keep = 0u;
                    const unsigned long long *cx = reinterpret_cast<const unsigned long long *>(&s_nxyz[0][jb * 32]);
                    const unsigned long long *cy = reinterpret_cast<const unsigned long long *>(&s_nxyz[1][jb * 32]);
                    const unsigned long long *cz = reinterpret_cast<const unsigned long long *>(&s_nxyz[2][jb * 32]);
#pragma unroll 4
                    for (int pp = 15; pp >= 0; --pp) {
                        const unsigned long long dx = f2_sub(xi2, cx[pp]);
                        const unsigned long long dy = f2_sub(yi2, cy[pp]);
                        const unsigned long long dz = f2_sub(zi2, cz[pp]);
                        unsigned long long s2 = f2_fma(dx, dx, nrc2);
                        s2 = f2_fma(dy, dy, s2);
                        s2 = f2_fma(dz, dz, s2);
                        keep = __funnelshift_l((unsigned)(s2 >> 32), keep, 1);  // slot 2pp+1
                        keep = __funnelshift_l((unsigned)s2, keep, 1);          // slot 2pp
                    }
                }
                keep = i < mh ? keep : 0u;
                if (diag && ib == jb) keep &= ~((2u << lane) - 1u);  // columns above the row
                const int c = __popc(keep);
                int rs = c;  // inclusive prefix of the row counts
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, rs, o);
                    if (lane >= o) rs += v;
                }
                const int total = __shfl_sync(0xffffffffu, rs, 31);
                rs -= c;  // exclusive: this row's first entry
                if (total == 0) continue;
                const unsigned col = transpose32(keep, lane);  // column `lane`: rows that keep it
                uint16_t *cl = s_cl[warp];
                Acc sx = Acc(0), sy = Acc(0), sz = Acc(0);  // j-side sums of column `lane`
                // ---- row passes of at most CAP survivors (one pass unless the item is dense)
                for (int r_lo = 0; r_lo < 32;) {
                    const int base = __shfl_sync(0xffffffffu, rs, r_lo);
                    const unsigned fit = __ballot_sync(0xffffffffu, lane >= r_lo && rs + c - base <= CAP);
                    const int r_hi = 32 - __clz(fit);  // rows r_lo .. r_hi-1 (rs is monotone)
                    const int nent = __shfl_sync(0xffffffffu, rs + c, r_hi - 1) - base;
                    const bool mine = lane >= r_lo && lane < r_hi;
                    // column `lane` restricted to the pass's rows, and its offset in
                    // column order
                    const unsigned prow = (r_hi == 32 ? ~0u : ((1u << r_hi) - 1u)) & ~((1u << r_lo) - 1u);
                    const unsigned cm = col & prow;
                    const int cc = __popc(cm);
                    int cs = cc;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, cs, o);
                        if (lane >= o) cs += v;
                    }
                    cs -= cc;
                    s_col[warp][lane] = cm;
                    s_cs[warp][lane] = cs;
                    // compaction: each row writes its survivors at its offset
                    if (mine) {
                        int pos = rs - base;
                        unsigned m = keep;
                        while (m) {
                            const int b = __ffs(m) - 1;
                            m &= m - 1;
                            q[pos++] = (uint16_t)((lane << 5) | b);
                        }
                    }
                    __syncwarp();
                    // force stage on full warps of survivors
                    for (int t0 = 0; t0 < nent; t0 += 32) {
                        const int t = t0 + lane;
                        const bool act = t < nent;
                        const uint16_t e = act ? q[t] : 0;
                        const int il = ib * 32 + (e >> 5), jl = jb * 32 + (e & 31);
                        const float4 pa = make_float4(s_hxyz[0][il], s_hxyz[1][il], s_hxyz[2][il], s_hq[il]);
                        const float4 pb = make_float4(s_nxyz[0][jl], s_nxyz[1][jl], s_nxyz[2][jl], s_nq[jl]);
                        float dx, dy, dz;
                        displacement<MI>(pa, pb, g, mb, dx, dy, dz);
                        const float r2 = pair_r2(dx, dy, dz);
                        const bool ok = act && (r2 < rc2);
                        const float2 ab = s_ab[s_ht[il] * T + s_nt[jl]];
                        const float kqq = __fmul_rn(kc, __fmul_rn(pa.w, pb.w));
                        float ir, ir2, ir6;
                        float f = pair_f(r2, ab.x, ab.y, kqq, ir, ir2, ir6);
                        f = ok ? f : 0.0f;
                        const float fx = __fmul_rn(f, dx), fy = __fmul_rn(f, dy), fz = __fmul_rn(f, dz);
                        if (act) {
                            // this pair's place in column order: column offset + rank of
                            // its row among the column's rows
                            const int k = e & 31, l = e >> 5;
                            cl[s_cs[warp][k] + __popc(s_col[warp][k] & ((1u << l) - 1u))] = (uint16_t)t;
                            if (MODE == MD_ACCUM_FIXED64) {
                                fb[0][t] = (Acc)(ok ? to_fixed(fx, a.status) : 0);
                                fb[1][t] = (Acc)(ok ? to_fixed(fy, a.status) : 0);
                                fb[2][t] = (Acc)(ok ? to_fixed(fz, a.status) : 0);
                            } else {
                                fb[0][t] = (Acc)fx;
                                fb[1][t] = (Acc)fy;
                                fb[2][t] = (Acc)fz;
                            }
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
                    __syncwarp();
                    // i-side: the row's survivors are contiguous
                    if (mine) {
                        const int p0 = rs - base;
                        for (int r = 0; r < c; ++r) {
                            ax += fb[0][p0 + r];
                            ay += fb[1][p0 + r];
                            az += fb[2][p0 + r];
                        }
                    }
                    // j-side (Newton's third law): column `lane` sums its entries, listed
                    // contiguously in column order
                    for (int r = 0; r < cc; ++r) {
                        const int p = cl[cs + r];
                        sx += fb[0][p];
                        sy += fb[1][p];
                        sz += fb[2][p];
                    }
                    __syncwarp();
                    r_lo = r_hi;
                }
                const int jt = jb * 32 + lane;
                smem_add<MODE>(&s_nf[0][jt], Acc(0) - sx);
                smem_add<MODE>(&s_nf[1][jt], Acc(0) - sy);
                smem_add<MODE>(&s_nf[2][jt], Acc(0) - sz);
            }
            if (cur_ib >= 0 && cur_ib * 32 + lane < mh) {
                const int ii = cur_ib * 32 + lane;
                smem_add<MODE>(&s_hf[0][ii], ax);
                smem_add<MODE>(&s_hf[1][ii], ay);
                smem_add<MODE>(&s_hf[2][ii], az);
            }
            __syncthreads();
            if (diag) {
                // the neighbour tile is the home tile: reactions join the home sums
                for (int t = threadIdx.x; t < mn; t += kHT) {
                    s_hf[0][t] += s_nf[0][t];
                    s_hf[1][t] += s_nf[1][t];
                    s_hf[2][t] += s_nf[2][t];
                }
            } else {
                // reactions of this tile -> global accumulators
                for (int t = threadIdx.x; t < mn; t += kHT) {
                    const int s = n_begin + n0 + t;
                    if (MODE == MD_ACCUM_FIXED64) {
                        unsigned long long *acc = static_cast<unsigned long long *>(a.accum);
                        atomicAdd(&acc[s], (unsigned long long)s_nf[0][t]);
                        atomicAdd(&acc[(size_t)a.n + s], (unsigned long long)s_nf[1][t]);
                        atomicAdd(&acc[2 * (size_t)a.n + s], (unsigned long long)s_nf[2][t]);
                    } else {
                        red_add_v4(static_cast<float4 *>(a.accum) + s, (float)s_nf[0][t],
                                   (float)s_nf[1][t], (float)s_nf[2][t]);
                    }
                }
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < mh; t += kHT) {
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
    Partial *mine = a.partials + (size_t)blockIdx.y * gridDim.x;
    block_partial<kHT>((double)e_lj, (double)e_c, (double)vir, cnt, mine);
    if (BATCHED && sys_pair_count && threadIdx.x == 0 && mine[blockIdx.x].count)
        atomicAdd(&sys_pair_count[sid], mine[blockIdx.x].count);
}

// Sorted-order accumulators -> forces_out in input order.
template <int MODE>
__global__ void __launch_bounds__(256)
k_finalize(const void *__restrict__ accum, const int32_t *__restrict__ perm, int n,
           void *__restrict__ forces_out, uint32_t *status)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int o = perm[s];
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

template <int MODE, bool ENERGY, bool MI, bool BATCHED = false, int W = kHWDefault,
          int CAP = KCap<MODE>::value>
void launch_half_t(const HalfArgs &h, dim3 grid, cudaStream_t stream, const BatchArgs &b = BatchArgs{},
                   unsigned long long *sys_pair_count = nullptr)
{
    using Acc = typename AccT<MODE>::T;
    const size_t dyn = sizeof(Acc) * W * 3 * CAP + sizeof(float2) * (size_t)h.ntypes * (size_t)h.ntypes;
    static const size_t dyn_max = sizeof(Acc) * W * 3 * CAP + sizeof(float2) * kMaxTypes * kMaxTypes;
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_half_shell<MODE, ENERGY, MI, BATCHED, W, CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)dyn_max);
    (void)attr;
    k_half_shell<MODE, ENERGY, MI, BATCHED, W, CAP><<<grid, W * 32, dyn, stream>>>(h, b, sys_pair_count);
}

// The half-shell shapes of the batched launches (md_batch_tuning): {warps per CTA,
// survivors buffered per warp} = 1 {4, default}, 2 {2, 256}, 3 {8, 256}, 4 {4, 128}.
// Shape 0 is the cluster kernel and 5 the cluster kernel on a persistent grid.
static_assert(MD_BATCH_SHAPES == 6, "one case per shape");

template <int MODE, bool MI>
void launch_batched_shape(int shape, const HalfArgs &h, dim3 grid, cudaStream_t stream,
                          const BatchArgs &b, unsigned long long *cnt)
{
    switch (shape) {
    case 2: launch_half_t<MODE, false, MI, true, 2, 256>(h, grid, stream, b, cnt); break;
    case 3: launch_half_t<MODE, false, MI, true, 8, 256>(h, grid, stream, b, cnt); break;
    case 4: launch_half_t<MODE, false, MI, true, 4, 128>(h, grid, stream, b, cnt); break;
    default: launch_half_t<MODE, false, MI, true, 4, KCap<MODE>::value>(h, grid, stream, b, cnt); break;
    }
}

}  // namespace

// Number of CTAs per home cell of the half-shell kernel.
int half_shell_pairs_per_cell(const BoxF &box)
{
    return (box.dims[0] < 3 || box.dims[1] < 3 || box.dims[2] < 3) ? 27 : 14;
}

// rc^2 of the exact test and the filter threshold rc'^2: the filter may see a
// difference short by |Llo| per wrapped axis and rounds differently from the exact
// test, so it is widened by that much and a few ulps.
void cutoff_thresholds(const BoxF &box, double rc, bool mi, float *rc2, float *rc2m)
{
    *rc2 = (float)(rc * rc);
    const double llo = fabs((double)box.Llo[0]) + fabs((double)box.Llo[1]) + fabs((double)box.Llo[2]);
    const double margin = mi ? 0.0 : 2.0 * rc * llo * 1.01 + 3.0 * llo * llo;
    *rc2m = (float)((double)*rc2 + margin + 8.0 * (double)*rc2 * 1.1920929e-7);
}

cudaError_t launch_forces_batched(const ForceArgs &a, const BatchArgs &b,
                                  unsigned long long *sys_pair_count, const WsLayout &ws,
                                  char *wsp, cudaStream_t stream, int shape_reg, int shape_mi)
{
    Partial *partials = reinterpret_cast<Partial *>(wsp + ws.partials);
    const size_t acc_bytes = (size_t)b.n * (fixed_output(a.mode) ? 24 : 16);
    // MD_ACCUM_FIXED_TILE runs on the cluster kernel only (shapes 0 and 5)
    if (a.mode == MD_ACCUM_FIXED_TILE && ((b.ncell_reg > 0 && shape_reg != 0 && shape_reg != 5) ||
                                          (b.ncell_mi > 0 && shape_mi != 0 && shape_mi != 5)))
        return cudaErrorInvalidValue;
    void *accum = wsp + ws.accum;
    cudaError_t e = a.accum_zeroed ? cudaSuccess : cudaMemsetAsync(accum, 0, acc_bytes, stream);
    if (e != cudaSuccess) return e;
    int *work = reinterpret_cast<int *>(wsp + ws.work);
    if (!a.accum_zeroed && (shape_reg == 5 || shape_mi == 5) &&
        (e = cudaMemsetAsync(work, 0, 2 * sizeof(int), stream)) != cudaSuccess)
        return e;
    // the batch's cells come from the fused MD-step build, already in cluster order;
    // both launches read them and accumulate in that order
    if (!a.presorted) return cudaErrorInvalidValue;
    HalfArgs h = {};
    h.cell_start = a.cell_start;
    h.pq = a.pos_q_sorted;
    h.ty = a.type_sorted;
    h.accum = accum;
    h.n = b.n;
    h.status = a.status;
    // the shared LJ table must hold the largest table of the batch
    h.ntypes = b.max_ntypes;
    if (h.ntypes < 1 || h.ntypes > kMaxTypes) return cudaErrorInvalidValue;
    if (b.ncell_reg > 0) {
        h.partials = partials;
        dim3 grid(b.ncell_reg, 14);
        if (shape_reg == 0 || shape_reg == 5)
            e = launch_cluster_batched(a.mode, false, b, a.cell_start, h.pq, h.ty, accum, partials,
                                       a.status, sys_pair_count, shape_reg == 5 ? work : nullptr, stream);
        else if (a.mode == MD_ACCUM_FIXED64) launch_batched_shape<MD_ACCUM_FIXED64, false>(shape_reg, h, grid, stream, b, sys_pair_count);
        else launch_batched_shape<MD_ACCUM_F32, false>(shape_reg, h, grid, stream, b, sys_pair_count);
        if (e != cudaSuccess) return e;
    }
    if (b.ncell_mi > 0) {
        h.partials = partials + (size_t)14 * b.ncell_reg;
        dim3 grid(b.ncell_mi, 27);
        if (shape_mi == 0 || shape_mi == 5)
            e = launch_cluster_batched(a.mode, true, b, a.cell_start, h.pq, h.ty, accum, h.partials,
                                       a.status, sys_pair_count, shape_mi == 5 ? work + 1 : nullptr, stream);
        else if (a.mode == MD_ACCUM_FIXED64) launch_batched_shape<MD_ACCUM_FIXED64, true>(shape_mi, h, grid, stream, b, sys_pair_count);
        else launch_batched_shape<MD_ACCUM_F32, true>(shape_mi, h, grid, stream, b, sys_pair_count);
        if (e != cudaSuccess) return e;
    }
    if ((e = launch_finalize_cluster(a, accum, ws, wsp, b.n, stream)) != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_half_shell(const ForceArgs &a, const WsLayout &ws, char *wsp, Partial *partials,
                              int *nblocks_out, cudaStream_t stream)
{
    const int per_cell = half_shell_pairs_per_cell(a.box);
    const bool mi = per_cell == 27;
    const size_t acc_bytes = (size_t)a.n * (a.mode == MD_ACCUM_FIXED64 ? 24 : 16);
    void *accum = wsp + ws.accum;
    cudaError_t e = cudaMemsetAsync(accum, 0, acc_bytes, stream);
    if (e != cudaSuccess) return e;
    HalfArgs h;
    h.cell_start = a.cell_start;
    h.pq = a.pos_q_sorted;
    h.ty = a.type_sorted;
    h.box = a.box;
    h.AB = a.AB;
    h.ntypes = a.ntypes;
    h.kc = a.k_coulomb;
    cutoff_thresholds(a.box, a.rc64, mi, &h.rc2, &h.rc2m);
    h.accum = accum;
    h.n = a.n;
    h.partials = partials;
    h.status = a.status;
    dim3 grid(a.box.ncell, per_cell);
    const bool en = a.energy_virial_out != nullptr;
    if (a.mode == MD_ACCUM_FIXED64) {
        if (mi) { if (en) launch_half_t<MD_ACCUM_FIXED64, true, true>(h, grid, stream); else launch_half_t<MD_ACCUM_FIXED64, false, true>(h, grid, stream); }
        else    { if (en) launch_half_t<MD_ACCUM_FIXED64, true, false>(h, grid, stream); else launch_half_t<MD_ACCUM_FIXED64, false, false>(h, grid, stream); }
        k_finalize<MD_ACCUM_FIXED64><<<(a.n + 255) / 256, 256, 0, stream>>>(accum, a.perm, a.n, a.forces_out, a.status);
    } else {
        if (mi) { if (en) launch_half_t<MD_ACCUM_F32, true, true>(h, grid, stream); else launch_half_t<MD_ACCUM_F32, false, true>(h, grid, stream); }
        else    { if (en) launch_half_t<MD_ACCUM_F32, true, false>(h, grid, stream); else launch_half_t<MD_ACCUM_F32, false, false>(h, grid, stream); }
        k_finalize<MD_ACCUM_F32><<<(a.n + 255) / 256, 256, 0, stream>>>(accum, a.perm, a.n, a.forces_out, a.status);
    }
    *nblocks_out = a.box.ncell * per_cell;
    return cudaGetLastError();
}

}  // namespace mdnb
