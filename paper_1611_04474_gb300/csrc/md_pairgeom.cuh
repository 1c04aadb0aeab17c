// md_pairgeom.cuh -- cell-pair geometry and accumulation helpers shared by the
// half-shell and cluster-pair force kernels (each translation unit gets its own copy).
//
// Periodic images: for an axis with >= 3 cells the neighbour cell's image is fixed by
// the stencil offset.  The box length L = Lhi + Llo (float + remainder); the coordinate
// next to the far face has Lhi subtracted when a tile is staged (exact, Sterbenz), and
// Llo is added to the difference in the force stage, so the displacement carries one
// rounding of its own size.  Boxes with an axis of 2 cells use the per-pair minimum
// image instead and enumerate each unordered cell pair once.
#pragma once

#include "md_internal.cuh"

namespace mdnb {
namespace {

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

// Launch order of the 14 half-shell pairs of a box with >= 3 cells per axis: the
// heaviest first (3 face neighbours, the cell itself, 6 edge neighbours, 4 corner
// neighbours; at the lattice density they hold about 390, 310, 185 and 70 cluster
// pairs in range), so that the last CTAs of a launch are the short ones.  Entry 0 is
// the cell itself, entry j >= 1 the forward neighbour kForward[j - 1].
__constant__ int kPairOrder[14] = {1, 3, 9, 0, 2, 4, 6, 8, 10, 12, 5, 7, 11, 13};

// Half-shell entry e (0: the cell itself, j >= 1: forward neighbour kForward[j - 1]) of
// home cell c in a box with >= 3 cells per axis; returns the wrap code of the neighbour
// (w_x + 3 w_y + 9 w_z + 13 with w_d in {-1, 0, 1} the face crossed along axis d; 13 for
// none), which fixes hs, ns and lo.
__device__ __forceinline__ int forward_pair(const BoxF &box, int c, int e, PairGeom &g)
{
    const int nx = box.dims[0], ny = box.dims[1];
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    g.home = c;
#pragma unroll
    for (int d = 0; d < 3; ++d) g.hs[d] = g.ns[d] = g.lo[d] = 0.0f;
    if (e == 0) {
        g.nbr = c;
        g.self = true;
        return 13;
    }
    int t[3] = {cx + kForward[e - 1][0], cy + kForward[e - 1][1], cz + kForward[e - 1][2]};
    int code = 13;
#pragma unroll
    for (int d = 0, m = 1; d < 3; ++d, m *= 3) {
        int w = 0;
        if (t[d] < 0) { t[d] += box.dims[d]; w = -1; }
        else if (t[d] >= box.dims[d]) { t[d] -= box.dims[d]; w = 1; }
        g.hs[d] = w > 0 ? box.Lhi[d] : 0.0f;
        g.ns[d] = w < 0 ? box.Lhi[d] : 0.0f;
        g.lo[d] = w > 0 ? -box.Llo[d] : (w < 0 ? box.Llo[d] : 0.0f);
        code += w * m;
    }
    g.nbr = t[0] + nx * (t[1] + ny * t[2]);
    g.self = false;
    return code;
}

// Cell pair number k of home cell c; false if k names no pair.
__device__ bool cell_pair(const BoxF &box, int c, int k, PairGeom &g)
{
    const int nx = box.dims[0], ny = box.dims[1], nz = box.dims[2];
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    if (!small_box(box)) {
        if (k < 0 || k > 13) return false;
        forward_pair(box, c, kPairOrder[k], g);
        return true;
    }
    g.home = c;
#pragma unroll
    for (int d = 0; d < 3; ++d) g.hs[d] = g.ns[d] = g.lo[d] = 0.0f;
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

// Box constants the per-pair minimum image needs.
struct MiBox {
    float Lhi[3], Llo[3], invL[3];
};

template <bool MI>
__device__ __forceinline__ void displacement(const float4 &pi, const float4 &pj, const PairGeom &g,
                                             const MiBox &box, float &dx, float &dy, float &dz)
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
// MD_ACCUM_FIXED_TILE sums in FP32 within a tile and rounds the partials to int64
template <>
struct AccT<MD_ACCUM_FIXED_TILE> {
    using T = float;
};

__device__ __forceinline__ void red_add_v4(float4 *addr, float a, float b, float c)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
                 "f"(c), "f"(0.0f)
                 : "memory");
}

// Packed FP32 pairs (Blackwell f32x2 ALU ops): two candidates per instruction.
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_dup(float x)
{
    // a register pair holding x twice (cheaper than a 64-bit shift and or)
    unsigned long long d;
    asm("mov.b64 %0, {%1, %1};" : "=l"(d) : "f"(x));
    return d;
}

}  // namespace
}  // namespace mdnb
