// md_step.cu -- pieces of the velocity-Verlet motion update around the force call (the
// paper's MD iteration: forces, then the atoms' motion, Sections I and II.A): the
// stand-alone half kick and the kinetic-energy log.  The drift, the wrap and the first
// half kick run fused with the cell build (md_cells.cu); the second half kick runs in
// the force kernels' last pass where it can.  State is FP64.
#include "md_internal.cuh"

namespace mdnb {
namespace {

constexpr int kThreads = 256;

// v += F ((dt/2) inv_mass 4.184e-4)
__global__ void __launch_bounds__(kThreads)
k_kick(double *__restrict__ vel, const void *__restrict__ forces, int mode,
       const float *__restrict__ inv_mass, int n, double half_dt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double f[3];
    load_force(forces, mode, i, f);
    const double kf = kick_factor((double)inv_mass[i], half_dt);
#pragma unroll
    for (int c = 0; c < 3; ++c) vel[3 * i + c] = kick_velocity(vel[3 * i + c], f[c], kf);
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
