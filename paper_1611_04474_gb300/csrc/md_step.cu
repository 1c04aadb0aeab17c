// md_step.cu -- velocity-Verlet motion update around the force call (the paper's MD
// iteration: forces, then the atoms' motion, Sections I and II.A).  State is FP64;
// the force kernels read a float copy of the wrapped positions that k_drift_wrap
// writes as (x, y, z, q).
#include "md_internal.cuh"

namespace mdnb {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void load_force(const void *forces, int mode, int i, double f[3])
{
    if (mode == MD_ACCUM_F32) {
        const float *F = static_cast<const float *>(forces);
        f[0] = F[3 * i];
        f[1] = F[3 * i + 1];
        f[2] = F[3 * i + 2];
    } else if (mode == MD_ACCUM_FIXED64) {
        const long long *F = static_cast<const long long *>(forces);
        const double s = 1.0 / 4294967296.0;
        f[0] = (double)F[3 * i] * s;
        f[1] = (double)F[3 * i + 1] * s;
        f[2] = (double)F[3 * i + 2] * s;
    } else {
        const double *F = static_cast<const double *>(forces);
        f[0] = F[3 * i];
        f[1] = F[3 * i + 1];
        f[2] = F[3 * i + 2];
    }
}

// v += (dt/2) * F * inv_mass * 4.184e-4
__global__ void __launch_bounds__(kThreads)
k_kick(double *__restrict__ vel, const void *__restrict__ forces, int mode,
       const float *__restrict__ inv_mass, int n, double half_dt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double f[3];
    load_force(forces, mode, i, f);
    double im = (double)inv_mass[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) vel[3 * i + c] += half_dt * f[c] * im * kAccelPerForcePerMass;
}

// x <- wrap(x + dt * v) in FP64; float copy (x, y, z, q) for the cell build and forces.
__global__ void __launch_bounds__(kThreads)
k_drift_wrap(double *__restrict__ pos, const double *__restrict__ vel, const float *__restrict__ q,
             int n, BoxF box, double dt, float4 *__restrict__ pos_q_out, uint32_t *status)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[3];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double v = pos[3 * i + c] + dt * vel[3 * i + c];
        if (isfinite(v)) {
            v = wrap_coord(v, box.L[c]);
        } else {
            ok = false;
        }
        x[c] = v;
        pos[3 * i + c] = v;
    }
    if (!ok) set_status(status, MD_STATUS_NONFINITE);
    pos_q_out[i] = make_float4((float)x[0], (float)x[1], (float)x[2], q[i]);
}

// The same for a batch: each atom wraps into its own system's box.
__global__ void __launch_bounds__(kThreads)
k_drift_wrap_batched(double *__restrict__ pos, const double *__restrict__ vel,
                     const float *__restrict__ q, BatchArgs b, double dt,
                     float4 *__restrict__ pos_q_out, uint32_t *status)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n) return;
    const BoxF &box = b.sys[b.atom_sys[i]].box;
    double x[3];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double v = pos[3 * i + c] + dt * vel[3 * i + c];
        if (isfinite(v)) {
            v = wrap_coord(v, box.L[c]);
        } else {
            ok = false;
        }
        x[c] = v;
        pos[3 * i + c] = v;
    }
    if (!ok) set_status(status, MD_STATUS_NONFINITE);
    pos_q_out[i] = make_float4((float)x[0], (float)x[1], (float)x[2], q[i]);
}

// Per-block kinetic energy 1/2 m v^2 (kcal/mol) into partials[blockIdx.x].e_lj.
__global__ void __launch_bounds__(kThreads)
k_kinetic(const double *__restrict__ vel, const float *__restrict__ inv_mass, int n,
          Partial *__restrict__ partials)
{
    __shared__ double s[kThreads];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (i < n) {
        double v2 = vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] + vel[3 * i + 2] * vel[3 * i + 2];
        ke = 0.5 * v2 / (double)inv_mass[i] / kAccelPerForcePerMass;
    }
    s[threadIdx.x] = ke;
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        Partial p = {s[0], 0.0, 0.0, 0ull};
        partials[blockIdx.x] = p;
    }
}

// Single block: row = {E_LJ, E_C, KE, W}, KE summed over the partials in a fixed order.
__global__ void __launch_bounds__(kThreads)
k_log_row(const Partial *__restrict__ partials, int nblocks, const double *__restrict__ ev,
          double *__restrict__ row)
{
    __shared__ double s[kThreads];
    double a = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += kThreads) a += partials[i].e_lj;
    s[threadIdx.x] = a;
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        row[0] = ev[0];
        row[1] = ev[1];
        row[2] = s[0];
        row[3] = ev[2];
    }
}

}  // namespace

cudaError_t launch_kick(double *vel, const void *forces, int mode, const float *inv_mass, int n,
                        double half_dt, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    k_kick<<<(n + kThreads - 1) / kThreads, kThreads, 0, stream>>>(vel, forces, mode, inv_mass, n,
                                                                   half_dt);
    return cudaGetLastError();
}

cudaError_t launch_drift_wrap(double *pos, const double *vel, const float *q, int n,
                              const BoxF &box, double dt, float4 *pos_q_out, uint32_t *status,
                              cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    k_drift_wrap<<<(n + kThreads - 1) / kThreads, kThreads, 0, stream>>>(pos, vel, q, n, box, dt,
                                                                         pos_q_out, status);
    return cudaGetLastError();
}

cudaError_t launch_drift_wrap_batched(double *pos, const double *vel, const float *q, const BatchArgs &b,
                                      double dt, float4 *pos_q_out, uint32_t *status,
                                      cudaStream_t stream)
{
    if (b.n <= 0) return cudaSuccess;
    k_drift_wrap_batched<<<(b.n + kThreads - 1) / kThreads, kThreads, 0, stream>>>(pos, vel, q, b, dt,
                                                                                  pos_q_out, status);
    return cudaGetLastError();
}

cudaError_t launch_energy_log_row(const double *vel, const float *inv_mass, int n,
                                  const double *energy_virial, double *row, const WsLayout &ws,
                                  char *wsp, cudaStream_t stream)
{
    Partial *partials = reinterpret_cast<Partial *>(wsp + ws.partials);
    int g = (n + kThreads - 1) / kThreads;
    if (g > ws.nslots) return cudaErrorInvalidValue;
    if (g > 0) k_kinetic<<<g, kThreads, 0, stream>>>(vel, inv_mass, n, partials);
    k_log_row<<<1, kThreads, 0, stream>>>(partials, g, energy_virial, row);
    return cudaGetLastError();
}

}  // namespace mdnb
