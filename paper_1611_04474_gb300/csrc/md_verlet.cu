// md_verlet.cu -- the passes of the MD step with a Verlet skin (md_step_verlet).
//
// The cell method of Section II.A rebuilds the cell list before every force evaluation.
// With a skin s, the cells (edge >= rc + s) and the order of the atoms within them (the
// cluster order of the force kernel) are kept while no atom has moved more than s/2 since
// they were built: every pair closer than rc then still lies in neighbouring kept cells
// (each of its atoms has moved less than s/2, and the cells are at least rc + s wide).  The
// force kernel reads the current positions through the kept order and filters cluster
// pairs on their current boxes, so only the binning and the ordering are saved.
//
//   k_verlet_drift  : half kick, drift, wrap (the arithmetic of the plain step), the
//                     float copy in input order, the accumulators zeroed, and the
//                     largest squared move since the last rebuild (one atomic max per
//                     block on the bits of a non-negative float)
//   k_verlet_decide : one thread: rebuild this step if the largest move exceeds s/2 (or
//                     when asked to), then clears the running maximum
// The rebuild kernels (md_cells.cu) and the force kernel read the decision on the device:
// no step waits for the host.
#include "md_internal.cuh"

namespace mdnb {
namespace {

constexpr int kDriftThreads = 256;

__global__ void __launch_bounds__(kDriftThreads)
k_verlet_drift(double *__restrict__ pos, double *__restrict__ vel, const void *__restrict__ forces,
               int mode, const float *__restrict__ inv_mass, const float *__restrict__ q, int n,
               BoxF box, double dt, double half_dt, int kick, float4 *__restrict__ pos_q,
               const float4 *__restrict__ x_ref, void *__restrict__ accum,
               VerletFlags *__restrict__ flags, uint32_t *status)
{
    __shared__ float s_max[kDriftThreads / 32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float d2 = 0.0f;
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
        pos_q[i] = p;
        // the move since the last rebuild, by the minimum image
        const float4 r = x_ref[i];
        const float dx = p.x - r.x, dy = p.y - r.y, dz = p.z - r.z;
        const float mx = dx - box.Lhi[0] * rintf(dx * box.invL[0]);
        const float my = dy - box.Lhi[1] * rintf(dy * box.invL[1]);
        const float mz = dz - box.Lhi[2] * rintf(dz * box.invL[2]);
        d2 = mx * mx + my * my + mz * mz;
        if (!(d2 >= 0.0f)) d2 = 3.0e38f;  // a non-finite position forces a rebuild
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = d2;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.0f;
#pragma unroll
        for (int w = 0; w < kDriftThreads / 32; ++w) m = fmaxf(m, s_max[w]);
        // non-negative floats order like their bit patterns
        atomicMax(&flags->maxdisp2, __float_as_uint(m));
    }
}

__global__ void k_verlet_decide(VerletFlags *flags, float threshold2, int force,
                                unsigned long long *rebuilds)
{
    if (threadIdx.x != 0) return;
    const float m = __uint_as_float(flags->maxdisp2);
    const int r = force || !(m <= threshold2);
    flags->rebuild = r;
    flags->maxdisp2 = 0u;
    if (r && rebuilds) *rebuilds += 1ull;
}

}  // namespace

cudaError_t launch_verlet_drift(double *pos, double *vel, const void *forces, int mode,
                                const float *inv_mass, const float *q, int n, const BoxF &box,
                                double dt, double half_dt, bool kick, float4 *pos_q,
                                const float4 *x_ref, void *accum, VerletFlags *flags,
                                uint32_t *status, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    const int g = (n + kDriftThreads - 1) / kDriftThreads;
    k_verlet_drift<<<g, kDriftThreads, 0, stream>>>(pos, vel, forces, mode, inv_mass, q, n, box, dt,
                                                    half_dt, kick ? 1 : 0, pos_q, x_ref, accum,
                                                    flags, status);
    return cudaGetLastError();
}

cudaError_t launch_verlet_decide(VerletFlags *flags, float threshold2, bool force,
                                 unsigned long long *rebuilds, cudaStream_t stream)
{
    k_verlet_decide<<<1, 32, 0, stream>>>(flags, threshold2, force ? 1 : 0, rebuilds);
    return cudaGetLastError();
}

}  // namespace mdnb
