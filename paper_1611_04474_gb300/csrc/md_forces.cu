// md_forces.cu -- short-range non-bonded forces, Eq. 1 (LJ) + Eq. 2 (Coulomb) under the
// cutoff of Section II.A, over the cell list (Algorithm 1).
//
// Full-shell kernel (MD_ALGO_FULL_SHELL): one CTA per home cell, one thread per home
// atom; the thread walks the distinct cells of the 3x3x3 stencil and every atom in
// them, filters r^2 < rc^2 and accumulates the force on its own atom only.  Each pair
// is evaluated from both sides, so no atomics are needed and every mode is
// deterministic.  This is Algorithm 1 as written, kept as the plain GPU baseline and
// as the path of the FP64 reference mode.
#include <math.h>

#include "md_internal.cuh"

namespace mdnb {

namespace {

constexpr int kFullThreads = 128;

// Distinct neighbour cells of home cell c (the 3x3x3 stencil names a cell more than
// once when an axis has fewer than three cells).
__device__ int stencil_cells(const BoxF &box, int c, int *out)
{
    int cx = c % box.dims[0], cy = (c / box.dims[0]) % box.dims[1], cz = c / (box.dims[0] * box.dims[1]);
    int m = 0;
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                int x = (cx + ox + box.dims[0]) % box.dims[0];
                int y = (cy + oy + box.dims[1]) % box.dims[1];
                int z = (cz + oz + box.dims[2]) % box.dims[2];
                int nb = x + box.dims[0] * (y + box.dims[1] * z);
                bool seen = false;
                for (int k = 0; k < m; ++k) seen |= (out[k] == nb);
                if (!seen) out[m++] = nb;
            }
    return m;
}

template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(kFullThreads)
k_full_shell(const int32_t *__restrict__ cell_start, const int32_t *__restrict__ perm,
             const float4 *__restrict__ pq, const int32_t *__restrict__ ty, BoxF box,
             const float2 *__restrict__ AB, int ntypes, float kc, double kc64, float rc2f,
             double rc2d, void *__restrict__ forces_out, Partial *__restrict__ partials,
             uint32_t *status)
{
    __shared__ float2 sAB[kMaxTypes * kMaxTypes];
    __shared__ int sNb[27];
    __shared__ int sNbCount;
    for (int t = threadIdx.x; t < ntypes * ntypes; t += kFullThreads) sAB[t] = AB[t];
    const int c = blockIdx.x;
    if (threadIdx.x == 0) sNbCount = stencil_cells(box, c, sNb);
    __syncthreads();
    const int nnb = sNbCount;
    const int a0 = cell_start[c], a1 = cell_start[c + 1];
    double e_lj = 0.0, e_c = 0.0, vir = 0.0;
    unsigned long long cnt = 0;

    for (int a = a0 + threadIdx.x; a < a1; a += kFullThreads) {
        const float4 pi = pq[a];
        const int ti = clamp_type(ty[a], ntypes, status);
        float fx = 0.f, fy = 0.f, fz = 0.f;
        long long ix = 0, iy = 0, iz = 0;
        double dx64 = 0.0, dy64 = 0.0, dz64 = 0.0;
        for (int k = 0; k < nnb; ++k) {
            const int nb = sNb[k];
            const int b0 = cell_start[nb], b1 = cell_start[nb + 1];
            for (int b = b0; b < b1; ++b) {
                if (b == a) continue;
                const float4 pj = pq[b];
                if (MODE == MD_ACCUM_F64) {
                    double dx = min_image_f64(pi.x, pj.x, box.L[0]);
                    double dy = min_image_f64(pi.y, pj.y, box.L[1]);
                    double dz = min_image_f64(pi.z, pj.z, box.L[2]);
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (!(r2 < rc2d)) continue;
                    const int tj = clamp_type(ty[b], ntypes, status);
                    const float2 ab = sAB[ti * ntypes + tj];
                    double kqq = kc64 * (double)pi.w * (double)pj.w;
                    double ir2 = 1.0 / r2;
                    double ir = sqrt(ir2);
                    double ir6 = ir2 * ir2 * ir2;
                    double ir8 = ir6 * ir2;
                    double f = (double)ab.x * ir8 * ir6 - (double)ab.y * ir8 + kqq * ir2 * ir;
                    dx64 += f * dx;
                    dy64 += f * dy;
                    dz64 += f * dz;
                    if (ENERGY) {
                        e_lj += 0.5 * ((double)ab.x / 12.0 * ir6 * ir6 - (double)ab.y / 6.0 * ir6);
                        e_c += 0.5 * kqq * ir;
                        vir += 0.5 * f * r2;
                    }
                } else {
                    float dx = min_image_f32(pi.x, pj.x, box.Lhi[0], box.Llo[0], box.invL[0]);
                    float dy = min_image_f32(pi.y, pj.y, box.Lhi[1], box.Llo[1], box.invL[1]);
                    float dz = min_image_f32(pi.z, pj.z, box.Lhi[2], box.Llo[2], box.invL[2]);
                    float r2 = pair_r2(dx, dy, dz);
                    if (!(r2 < rc2f)) continue;
                    const int tj = clamp_type(ty[b], ntypes, status);
                    const float2 ab = sAB[ti * ntypes + tj];
                    float kqq = __fmul_rn(kc, __fmul_rn(pi.w, pj.w));
                    float ir, ir2, ir6;
                    float f = pair_f(r2, ab.x, ab.y, kqq, ir, ir2, ir6);
                    float Fx = __fmul_rn(f, dx), Fy = __fmul_rn(f, dy), Fz = __fmul_rn(f, dz);
                    if (MODE == MD_ACCUM_FIXED64) {
                        ix += to_fixed(Fx, status);
                        iy += to_fixed(Fy, status);
                        iz += to_fixed(Fz, status);
                    } else {
                        fx += Fx;
                        fy += Fy;
                        fz += Fz;
                    }
                    if (ENERGY) {
                        e_lj += 0.5 * (double)pair_u_lj(ab.x, ab.y, ir6);
                        e_c += 0.5 * (double)(kqq * ir);
                        vir += 0.5 * (double)(f * r2);
                    }
                }
                cnt += (b > a);
            }
        }
        const int o = perm[a];
        if (MODE == MD_ACCUM_F64) {
            double *F = static_cast<double *>(forces_out);
            F[3 * o + 0] = dx64;
            F[3 * o + 1] = dy64;
            F[3 * o + 2] = dz64;
            if (!isfinite(dx64 + dy64 + dz64)) set_status(status, MD_STATUS_NONFINITE);
        } else if (MODE == MD_ACCUM_FIXED64) {
            long long *F = static_cast<long long *>(forces_out);
            F[3 * o + 0] = ix;
            F[3 * o + 1] = iy;
            F[3 * o + 2] = iz;
        } else {
            float *F = static_cast<float *>(forces_out);
            F[3 * o + 0] = fx;
            F[3 * o + 1] = fy;
            F[3 * o + 2] = fz;
            if (!isfinite(fx + fy + fz)) set_status(status, MD_STATUS_NONFINITE);
        }
    }
    block_partial<kFullThreads>(e_lj, e_c, vir, cnt, partials);
}

}  // namespace

// Single block: fixed-order sum of the per-block partials.
__global__ void __launch_bounds__(256)
k_reduce_partials(const Partial *__restrict__ partials, int nblocks,
                  double *__restrict__ energy_virial_out, unsigned long long *__restrict__ count_out)
{
    __shared__ double s[3][256];
    __shared__ unsigned long long sc[256];
    double a = 0.0, b = 0.0, c = 0.0;
    unsigned long long k = 0;
    for (int i = threadIdx.x; i < nblocks; i += 256) {
        Partial p = partials[i];
        a += p.e_lj;
        b += p.e_c;
        c += p.w;
        k += p.count;
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    s[2][threadIdx.x] = c;
    sc[threadIdx.x] = k;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s[0][threadIdx.x] += s[0][threadIdx.x + h];
            s[1][threadIdx.x] += s[1][threadIdx.x + h];
            s[2][threadIdx.x] += s[2][threadIdx.x + h];
            sc[threadIdx.x] += sc[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (energy_virial_out) {
            energy_virial_out[0] = s[0][0];
            energy_virial_out[1] = s[1][0];
            energy_virial_out[2] = s[2][0];
        }
        if (count_out) *count_out = sc[0];
    }
}

template <int MODE, bool ENERGY>
static void launch_full(const ForceArgs &a, Partial *partials, cudaStream_t stream)
{
    float rc2f = (float)(a.rc64 * a.rc64);
    double rc2d = a.rc64 * a.rc64;
    k_full_shell<MODE, ENERGY><<<a.box.ncell, kFullThreads, 0, stream>>>(
        a.cell_start, a.perm, a.pos_q_sorted, a.type_sorted, a.box, a.AB, a.ntypes, a.k_coulomb,
        a.k_coulomb64, rc2f, rc2d, a.forces_out, partials, a.status);
}

cudaError_t launch_forces(const ForceArgs &a, const WsLayout &ws, char *wsp, cudaStream_t stream)
{
    Partial *partials = reinterpret_cast<Partial *>(wsp + ws.partials);
    const bool energy = a.energy_virial_out != nullptr;
    if (a.n == 0) {
        // nothing to evaluate: zero outputs
        if (a.energy_virial_out) cudaMemsetAsync(a.energy_virial_out, 0, 3 * sizeof(double), stream);
        if (a.pair_count_out) cudaMemsetAsync(a.pair_count_out, 0, sizeof(unsigned long long), stream);
        return cudaGetLastError();
    }
    // the FP64 reference mode always runs the full-shell kernel
    int algo = a.algo;
    if (algo == MD_ALGO_DEFAULT || a.mode == MD_ACCUM_F64)
        algo = a.mode == MD_ACCUM_F64 ? MD_ALGO_FULL_SHELL : MD_ALGO_CLUSTER;
    // MD_ACCUM_FIXED_TILE exists in the cluster kernel only (the ABI rejects other kernels)
    if (a.mode == MD_ACCUM_FIXED_TILE && algo != MD_ALGO_CLUSTER) return cudaErrorInvalidValue;
    int nblocks = a.box.ncell;
    if (algo == MD_ALGO_CLUSTER) {
        cudaError_t e = launch_cluster(a, ws, wsp, partials, &nblocks, stream);
        if (e != cudaSuccess) return e;
    } else if (algo == MD_ALGO_HALF_SHELL) {
        cudaError_t e = launch_half_shell(a, ws, wsp, partials, &nblocks, stream);
        if (e != cudaSuccess) return e;
    } else {
        switch (a.mode * 2 + (energy ? 1 : 0)) {
        case MD_ACCUM_F32 * 2 + 0: launch_full<MD_ACCUM_F32, false>(a, partials, stream); break;
        case MD_ACCUM_F32 * 2 + 1: launch_full<MD_ACCUM_F32, true>(a, partials, stream); break;
        case MD_ACCUM_FIXED64 * 2 + 0: launch_full<MD_ACCUM_FIXED64, false>(a, partials, stream); break;
        case MD_ACCUM_FIXED64 * 2 + 1: launch_full<MD_ACCUM_FIXED64, true>(a, partials, stream); break;
        case MD_ACCUM_F64 * 2 + 0: launch_full<MD_ACCUM_F64, false>(a, partials, stream); break;
        case MD_ACCUM_F64 * 2 + 1: launch_full<MD_ACCUM_F64, true>(a, partials, stream); break;
        default: return cudaErrorInvalidValue;
        }
    }
    if (a.energy_virial_out || a.pair_count_out)
        k_reduce_partials<<<1, 256, 0, stream>>>(partials, nblocks, a.energy_virial_out,
                                                 a.pair_count_out);
    // the half kick of an MD step: inside the cluster kernel's finalize, else here
    if (a.kick_vel && algo != MD_ALGO_CLUSTER) {
        cudaError_t e = launch_kick(a.kick_vel, a.forces_out, a.mode, a.kick_inv_mass, a.n, a.kick_half_dt, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace mdnb
