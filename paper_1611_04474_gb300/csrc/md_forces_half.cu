// md_forces_half.cu -- half-shell cell-pair force kernel (MD_ALGO_HALF_SHELL).
//
// The loop nest of Algorithm 1 with every unordered pair met once: each CTA takes one
// (home cell, neighbour cell) pair of the half shell (the home cell itself with i<j,
// plus 13 forward neighbours), and the reaction -F goes to the neighbour atom
// (Newton's third law).  The two stages of the paper's enhanced accelerator
// (Section V.B: cheap distance filters feeding one expensive force unit through a
// FIFO) become, inside one warp:
//   filter:  32 home atoms (one per lane) x 32 neighbour atoms (broadcast from shared
//            memory); each lane folds the sign of rc'^2 - r^2 of its 32 candidates
//            into a bit mask with one funnel shift per candidate;
//   compact: popcount + warp prefix sum place the surviving (i, j) pairs in a per-warp
//            queue in shared memory;
//   force:   full warps of 32 survivors evaluate Eq. 1 + Eq. 2, so a low survival rate
//            does not idle lanes of the force math.  The exact test r^2 < rc^2 is
//            applied here; the filter uses rc'^2 = rc^2 + a tiny margin so that it
//            never rejects a pair the exact test keeps.
// Forces on both atoms of a pair are summed in shared memory per tile, then added to
// sorted-order accumulators in global memory with one vector atomic per atom per tile.
//
// Periodic images: for an axis with >= 3 cells the neighbour cell's image is fixed by
// the stencil offset.  The box length L = Lhi + Llo (float + remainder); the coordinate
// next to the far face has Lhi subtracted when the tile is staged (exact, Sterbenz),
// and Llo is added to the difference in the force stage, so the displacement carries
// one rounding of its own size.  Boxes with an axis of 2 cells use the per-pair
// minimum image instead and enumerate each unordered cell pair once.
#include <math.h>

#include "md_internal.cuh"

namespace mdnb {
namespace {

constexpr int kHW = 4;               // warps per CTA
constexpr int kHT = kHW * 32;        // threads per CTA
constexpr int kTile = 256;           // atoms of a cell staged at once (i, j indices fit 8 bits)
constexpr int kQCap = 1024 + 64;     // survivor queue per warp: one 32x32 item + leftovers
constexpr float kFar = 1.0e18f;      // coordinate of padding slots: fails every filter

__constant__ int kForward[13][3] = {{1, 0, 0},   {-1, 1, 0}, {0, 1, 0},  {1, 1, 0},  {-1, -1, 1},
                                    {0, -1, 1},  {1, -1, 1}, {-1, 0, 1}, {0, 0, 1},  {1, 0, 1},
                                    {-1, 1, 1},  {0, 1, 1},  {1, 1, 1}};

struct PairGeom {
    int home, nbr;
    bool self;
    float hs[3];  // subtracted from home coordinates
    float ns[3];  // subtracted from neighbour coordinates
    float lo[3];  // added to the difference
};

__device__ __forceinline__ bool small_box(const BoxF &b)
{
    return b.dims[0] < 3 || b.dims[1] < 3 || b.dims[2] < 3;
}

// Cell pair number k of home cell c; false if k names no pair.
__device__ bool cell_pair(const BoxF &box, int c, int k, PairGeom &g)
{
    const int nx = box.dims[0], ny = box.dims[1], nz = box.dims[2];
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    g.home = c;
#pragma unroll
    for (int d = 0; d < 3; ++d) g.hs[d] = g.ns[d] = g.lo[d] = 0.0f;
    if (!small_box(box)) {
        if (k == 0) {
            g.nbr = c;
            g.self = true;
            return true;
        }
        if (k > 13) return false;
        int t[3] = {cx + kForward[k - 1][0], cy + kForward[k - 1][1], cz + kForward[k - 1][2]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int w = 0;
            if (t[d] < 0) { t[d] += box.dims[d]; w = -1; }
            else if (t[d] >= box.dims[d]) { t[d] -= box.dims[d]; w = 1; }
            g.hs[d] = w > 0 ? box.Lhi[d] : 0.0f;
            g.ns[d] = w < 0 ? box.Lhi[d] : 0.0f;
            g.lo[d] = w > 0 ? -box.Llo[d] : (w < 0 ? box.Llo[d] : 0.0f);
        }
        g.nbr = t[0] + nx * (t[1] + ny * t[2]);
        g.self = false;
        return true;
    }
    // small box: distinct cells of the 27-stencil, each unordered pair once (c' > c)
    if (k > 26) return false;
    auto cell_of = [&](int kk) {
        int ox = kk % 3 - 1, oy = (kk / 3) % 3 - 1, oz = kk / 9 - 1;
        int x = (cx + ox + nx) % nx, y = (cy + oy + ny) % ny, z = (cz + oz + nz) % nz;
        return x + nx * (y + ny * z);
    };
    if (k == 13) {
        g.nbr = c;
        g.self = true;
        return true;
    }
    int nb = cell_of(k);
    if (nb <= c) return false;
    for (int kk = 0; kk < k; ++kk)
        if (cell_of(kk) == nb) return false;
    g.nbr = nb;
    g.self = false;
    return true;
}

template <bool MI>
__device__ __forceinline__ void displacement(const float4 &pi, const float4 &pj, const PairGeom &g,
                                             const BoxF &box, float &dx, float &dy, float &dz)
{
    if (MI) {
        dx = min_image_f32(pi.x, pj.x, box.Lhi[0], box.Llo[0], box.invL[0]);
        dy = min_image_f32(pi.y, pj.y, box.Lhi[1], box.Llo[1], box.invL[1]);
        dz = min_image_f32(pi.z, pj.z, box.Lhi[2], box.Llo[2], box.invL[2]);
    } else {
        dx = (pi.x - pj.x) + g.lo[0];
        dy = (pi.y - pj.y) + g.lo[1];
        dz = (pi.z - pj.z) + g.lo[2];
    }
}

template <int MODE>
struct AccT;
template <>
struct AccT<MD_ACCUM_F32> {
    using T = float;
};
template <>
struct AccT<MD_ACCUM_FIXED64> {
    using T = unsigned long long;
};

__device__ __forceinline__ void red_add_v4(float4 *addr, float a, float b, float c)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
                 "f"(c), "f"(0.0f)
                 : "memory");
}

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

template <int MODE, bool ENERGY, bool MI>
__global__ void __launch_bounds__(kHT, 4) k_half_shell(HalfArgs a)
{
    using Acc = typename AccT<MODE>::T;
    __shared__ float4 s_hp[kTile];
    __shared__ float4 s_np[kTile];
    __shared__ int s_ht[kTile];
    __shared__ int s_nt[kTile];
    __shared__ Acc s_hf[3][kTile];
    __shared__ Acc s_nf[3][kTile];
    __shared__ uint16_t s_q[kHW][kQCap];
    __shared__ float2 s_ab[kMaxTypes * kMaxTypes];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int T = a.ntypes;
    float e_lj = 0.f, e_c = 0.f, vir = 0.f;
    unsigned long long cnt = 0;

    PairGeom g;
    const bool valid = cell_pair(a.box, blockIdx.x, blockIdx.y, g);
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
    for (int t = threadIdx.x; t < T * T; t += kHT) s_ab[t] = a.AB[t];
    uint16_t *q = s_q[warp];

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
            s_hp[t] = p;
            s_ht[t] = ty;
            s_hf[0][t] = s_hf[1][t] = s_hf[2][t] = Acc(0);
        }
        for (int n0 = g.self ? h0 : 0; n0 < nn; n0 += kTile) {
            const int mn = min(kTile, nn - n0);
            const bool diag = g.self && n0 == h0;
            const int mn32 = (mn + 31) & ~31;
            __syncthreads();
            if (!diag) {
                for (int t = threadIdx.x; t < mn32; t += kHT) {
                    float4 p;
                    int ty = 0;
                    if (t < mn) {
                        p = a.pq[n_begin + n0 + t];
                        p.x -= g.ns[0];
                        p.y -= g.ns[1];
                        p.z -= g.ns[2];
                        ty = clamp_type(a.ty[n_begin + n0 + t], T, a.status);
                    } else {
                        p = make_float4(kFar, kFar, kFar, 0.f);
                    }
                    s_np[t] = p;
                    s_nt[t] = ty;
                    s_nf[0][t] = s_nf[1][t] = s_nf[2][t] = Acc(0);
                }
            }
            __syncthreads();
            const float4 *np = diag ? s_hp : s_np;
            const int *nt = diag ? s_ht : s_nt;
            Acc(*nf)[kTile] = diag ? s_hf : s_nf;

            // one batch of 32 queued survivors through the force math
            auto force_batch = [&](int base, int count) {
                const bool act = lane < count;
                const uint16_t e = act ? q[base + lane] : 0;
                const int il = e >> 8, jl = e & 255;
                const float4 pi = s_hp[il], pj = np[jl];
                float dx, dy, dz;
                displacement<MI>(pi, pj, g, a.box, dx, dy, dz);
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const bool ok = act && (r2 < a.rc2);
                const float2 ab = s_ab[s_ht[il] * T + nt[jl]];
                const float kqq = a.kc * pi.w * pj.w;
                const float ir2 = __frcp_rn(r2);
                const float ir = rsqrtf(r2);
                const float ir6 = ir2 * ir2 * ir2;
                const float ir8 = ir6 * ir2;
                float f = ab.x * (ir8 * ir6) - ab.y * ir8 + kqq * ir2 * ir;
                f = ok ? f : 0.0f;
                const float fx = f * dx, fy = f * dy, fz = f * dz;
                if (ok) {
                    if (MODE == MD_ACCUM_FIXED64) {
                        unsigned long long tx = (unsigned long long)to_fixed(fx, a.status);
                        unsigned long long ty_ = (unsigned long long)to_fixed(fy, a.status);
                        unsigned long long tz = (unsigned long long)to_fixed(fz, a.status);
                        atomicAdd((unsigned long long *)&s_hf[0][il], tx);
                        atomicAdd((unsigned long long *)&s_hf[1][il], ty_);
                        atomicAdd((unsigned long long *)&s_hf[2][il], tz);
                        atomicAdd((unsigned long long *)&nf[0][jl], 0ull - tx);
                        atomicAdd((unsigned long long *)&nf[1][jl], 0ull - ty_);
                        atomicAdd((unsigned long long *)&nf[2][jl], 0ull - tz);
                    } else {
                        atomicAdd((float *)&s_hf[0][il], fx);
                        atomicAdd((float *)&s_hf[1][il], fy);
                        atomicAdd((float *)&s_hf[2][il], fz);
                        atomicAdd((float *)&nf[0][jl], -fx);
                        atomicAdd((float *)&nf[1][jl], -fy);
                        atomicAdd((float *)&nf[2][jl], -fz);
                    }
                    cnt += 1;
                    if (ENERGY) {
                        e_lj += ab.x * (1.0f / 12.0f) * (ir6 * ir6) - ab.y * (1.0f / 6.0f) * ir6;
                        e_c += kqq * ir;
                        vir += f * r2;
                    }
                }
            };

            const int nib = mh32 >> 5, njb = mn32 >> 5;
            const int nitems = diag ? nib * (nib + 1) / 2 : nib * njb;
            int qn = 0;
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
                const float4 pi = s_hp[i];
                unsigned fail = 0u;
#pragma unroll 8
                for (int jj = 0; jj < 32; ++jj) {
                    const float4 pj = np[jb * 32 + jj];
                    float s;
                    if (MI) {
                        float dx, dy, dz;
                        displacement<true>(pi, pj, g, a.box, dx, dy, dz);
                        s = fmaf(-dz, dz, fmaf(-dy, dy, fmaf(-dx, dx, a.rc2m)));
                    } else {
                        const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
                        s = fmaf(-dz, dz, fmaf(-dy, dy, fmaf(-dx, dx, a.rc2m)));
                    }
                    // (fail << 1) | sign(s): a negative s rejects the candidate
                    fail = __funnelshift_l(__float_as_uint(s), fail, 1);
                }
                // bit b of keep <-> neighbour slot jb*32 + 31 - b
                unsigned keep = i < mh ? ~fail : 0u;  // padding lanes keep nothing
                if (diag && ib == jb) keep &= lane == 31 ? 0u : ((1u << (31 - lane)) - 1u);
                const int c = __popc(keep);
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                int pos = qn + incl - c;
                const uint16_t ibase = (uint16_t)(i << 8);
                const int jtop = jb * 32 + 31;
                unsigned m = keep;
                while (m) {
                    const int b = __ffs(m) - 1;
                    m &= m - 1;
                    q[pos++] = (uint16_t)(ibase | (jtop - b));
                }
                __syncwarp();
                qn += total;
                int done = 0;
                while (qn - done >= 32) {
                    force_batch(done, 32);
                    done += 32;
                }
                if (done > 0) {
                    const int rem = qn - done;
                    const uint16_t v = lane < rem ? q[done + lane] : 0;
                    __syncwarp();
                    if (lane < rem) q[lane] = v;
                    __syncwarp();
                    qn = rem;
                }
            }
            if (qn > 0) force_batch(0, qn);
            __syncthreads();
            if (!diag) {
                // reactions on the neighbour tile -> global accumulators
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
    block_partial<kHT>((double)e_lj, (double)e_c, (double)vir, cnt,
                       a.partials + (size_t)blockIdx.y * gridDim.x);
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

template <int MODE, bool ENERGY, bool MI>
void launch_half_t(const HalfArgs &h, dim3 grid, cudaStream_t stream)
{
    k_half_shell<MODE, ENERGY, MI><<<grid, kHT, 0, stream>>>(h);
}

}  // namespace

// Number of CTAs per home cell of the half-shell kernel.
int half_shell_pairs_per_cell(const BoxF &box)
{
    return (box.dims[0] < 3 || box.dims[1] < 3 || box.dims[2] < 3) ? 27 : 14;
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
    const float rc2 = (float)(a.rc64 * a.rc64);
    // the filter may see a difference short by |Llo| per wrapped axis and rounds
    // differently from the exact test: widen it by that much and a few ulps
    const double llo = fabs((double)a.box.Llo[0]) + fabs((double)a.box.Llo[1]) + fabs((double)a.box.Llo[2]);
    const double margin = mi ? 0.0 : 2.0 * a.rc64 * llo * 1.01 + 3.0 * llo * llo;
    h.rc2 = rc2;
    h.rc2m = (float)((double)rc2 + margin + 8.0 * (double)rc2 * 1.1920929e-7);
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
