// md_abi.cu -- the extern "C" entry points declared in include/md_nonbonded.h:
// argument validation, workspace layout, and the order of kernel launches.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "md_internal.cuh"

namespace mdnb {

namespace {
constexpr int kMaxCells = 1 << 24;
constexpr int kMaxAtoms = (1 << 30);
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

int validate_box(const double *L)
{
    if (!L) return MD_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(L[d] > 0.0) || !isfinite(L[d])) return MD_ERR_INVALID_ARG;
    return MD_OK;
}

int compute_dims(const double *L, double rc, int32_t *dims)
{
    int e = validate_box(L);
    if (e) return e;
    if (!(rc > 0.0) || !isfinite(rc)) return MD_ERR_CUTOFF;
    double lmin = fmin(L[0], fmin(L[1], L[2]));
    if (!(rc < 0.5 * lmin)) return MD_ERR_CUTOFF;
    long long prod = 1;
    for (int d = 0; d < 3; ++d) {
        double nd = floor(L[d] / rc);
        if (nd > (double)kMaxCells) return MD_ERR_TOO_LARGE;
        dims[d] = nd < 1.0 ? 1 : (int32_t)nd;
        prod *= dims[d];
    }
    if (prod > kMaxCells) return MD_ERR_TOO_LARGE;
    return MD_OK;
}

int check_dims(const int32_t *dims, int *ncell)
{
    if (!dims) return MD_ERR_INVALID_ARG;
    long long prod = 1;
    for (int d = 0; d < 3; ++d) {
        if (dims[d] < 1) return MD_ERR_INVALID_ARG;
        prod *= dims[d];
        if (prod > kMaxCells) return MD_ERR_TOO_LARGE;
    }
    *ncell = (int)prod;
    return MD_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Returns the 256-byte aligned start of the caller's workspace or nullptr.
char *ws_base(void *workspace, size_t ws_bytes, const WsLayout &ws)
{
    if (!workspace) return nullptr;
    uintptr_t p = reinterpret_cast<uintptr_t>(workspace);
    uintptr_t a = (p + kAlign - 1) & ~(uintptr_t)(kAlign - 1);
    if (ws_bytes < (a - p) + ws.total) return nullptr;
    return reinterpret_cast<char *>(a);
}

int cuda_code(cudaError_t e) { return e == cudaSuccess ? MD_OK : MD_ERR_CUDA; }

int check_ff(const md_forcefield *ff)
{
    if (!ff || !ff->AB) return MD_ERR_INVALID_ARG;
    if (ff->ntypes < 1 || ff->ntypes > kMaxTypes) return MD_ERR_INVALID_ARG;
    if (!isfinite(ff->k_coulomb)) return MD_ERR_INVALID_ARG;
    if (!aligned16(ff->AB) && (reinterpret_cast<uintptr_t>(ff->AB) & 7u)) return MD_ERR_INVALID_ARG;
    return MD_OK;
}
}  // namespace

BoxF make_box(const double *L, const int32_t *dims)
{
    BoxF b;
    long long prod = 1;
    for (int d = 0; d < 3; ++d) {
        b.L[d] = L[d];
        b.Lhi[d] = (float)L[d];
        b.Llo[d] = (float)(L[d] - (double)b.Lhi[d]);
        b.invL[d] = (float)(1.0 / L[d]);
        b.inv_edge[d] = (double)dims[d] / L[d];
        b.Lin[d] = (float)L[d];
        if ((double)b.Lin[d] > L[d]) b.Lin[d] = nextafterf(b.Lin[d], 0.0f);
        b.inv_edge_f[d] = (float)b.inv_edge[d];
        b.dims[d] = dims[d];
        prod *= dims[d];
    }
    b.ncell = (int)prod;
    return b;
}

int bin_capacity(int n, int ncell)
{
    const long long mean = ((long long)n + ncell - 1) / (ncell > 0 ? ncell : 1);
    const long long cap = (2 * mean + 64 + 31) / 32 * 32;
    return (int)(cap < (1LL << 30) ? cap : (1LL << 30));
}

// Whether a cell grid has an axis of 2 cells (or fewer): per-pair minimum image.
static bool split_dims(const int32_t *d)
{
    return d[0] < 3 || d[1] < 3 || d[2] < 3;
}

WsLayout ws_layout(int n, int ncell, bool bins, bool verlet, bool split)
{
    WsLayout w;
    size_t nn = (size_t)(n > 0 ? n : 1);
    size_t nc = (size_t)(ncell > 0 ? ncell : 1);
    // one partial per CTA of a cell-pair kernel at most
    int slots = 27 * (split ? kMiSplit : 1) * ncell;
    int kin = (int)((nn + 255) / 256);
    if (slots < kin) slots = kin;
    if (slots < 2048) slots = 2048;
    w.nslots = slots;
    size_t off = 0;
    w.cell_id = off;         off = align_up(off + sizeof(int32_t) * nn);
    w.cell_cnt = off;        off = align_up(off + sizeof(int32_t) * (nc + 1));
    w.perm_tmp = off;        off = align_up(off + sizeof(int32_t) * nn);
    w.accum = off;           off = align_up(off + 32 * nn);
    w.partials = off;        off = align_up(off + sizeof(Partial) * (size_t)slots);
    w.ev = off;              off = align_up(off + 4 * sizeof(double));
    w.st_cell_start = off;   off = align_up(off + sizeof(int32_t) * (nc + 1));
    w.st_perm = off;         off = align_up(off + sizeof(int32_t) * nn);
    w.st_pos_q_sorted = off; off = align_up(off + sizeof(float4) * nn);
    w.st_type_sorted = off;  off = align_up(off + sizeof(int32_t) * nn);
    w.st_pos_q = off;        off = align_up(off + sizeof(float4) * nn);
    w.clu_pos_q = off;       off = align_up(off + sizeof(float4) * nn);
    w.clu_type = off;        off = align_up(off + sizeof(int32_t) * nn);
    w.clu_order = off;       off = align_up(off + sizeof(int32_t) * nn);
    w.clu_box = off;         off = align_up(off + 2 * sizeof(float4) * nn);
    w.work = off;            off = align_up(off + 2 * sizeof(int32_t));
    w.bin_cap = bins && n > 0 ? bin_capacity(n, (int)nc) : 0;
    w.bins = off;            off = align_up(off + sizeof(int32_t) * nc * (size_t)w.bin_cap);
    w.v_ref = off;           off = align_up(off + (verlet ? sizeof(float4) * nn : 0));
    w.v_flags = off;         off = align_up(off + (verlet ? sizeof(VerletFlags) : 0));
    w.total = off;
    return w;
}

// Batch layout on the host: per-system cells and the scratch of the whole batch.
static int batch_layout(int32_t nsys, const md_system_desc *systems, BatchLayout *bl,
                        std::vector<int32_t> *dims_out)
{
    if (nsys < 1 || !systems) return MD_ERR_INVALID_ARG;
    long long n = 0, ncell = 0, ncell_mi = 0;
    dims_out->resize(3 * (size_t)nsys);
    for (int s = 0; s < nsys; ++s) {
        const md_system_desc &d = systems[s];
        if (d.n < 0) return MD_ERR_INVALID_ARG;
        int e = check_ff(&d.ff);
        if (e) return e;
        int32_t *dims = dims_out->data() + 3 * s;
        if ((e = compute_dims(d.box_L, d.ff.rc, dims))) return e;
        long long nc = (long long)dims[0] * dims[1] * dims[2];
        n += d.n;
        ncell += nc;
        if (dims[0] < 3 || dims[1] < 3 || dims[2] < 3) ncell_mi += nc;
    }
    if (n > kMaxAtoms || ncell > kMaxCells) return MD_ERR_TOO_LARGE;
    bl->nsys = nsys;
    bl->n = (int)n;
    bl->ncell = (int)ncell;
    bl->ncell_mi = (int)ncell_mi;
    bl->ncell_reg = (int)(ncell - ncell_mi);
    size_t off = 0;
    bl->sys = off;       off = align_up(off + sizeof(SysDesc) * (size_t)nsys);
    bl->cell_sys = off;  off = align_up(off + sizeof(int) * (size_t)ncell);
    bl->cell_list = off; off = align_up(off + sizeof(int) * (size_t)ncell);
    bl->atom_sys = off;  off = align_up(off + sizeof(int) * (size_t)(n > 0 ? n : 1));
    bl->run = ws_layout((int)n, (int)ncell, false, false, ncell_mi > 0);
    bl->run_base = off;
    bl->total = off + bl->run.total;
    return MD_OK;
}

}  // namespace mdnb

using namespace mdnb;

extern "C" {

const char *md_strerror(int code)
{
    switch (code) {
    case MD_OK: return "ok";
    case MD_ERR_INVALID_ARG: return "invalid argument";
    case MD_ERR_CUTOFF: return "cutoff must satisfy 0 < rc < min(L)/2 and match the cell dims";
    case MD_ERR_WORKSPACE: return "workspace missing or smaller than md_workspace_bytes";
    case MD_ERR_CUDA: return "CUDA launch or asynchronous call failed";
    case MD_ERR_TOO_LARGE: return "too many atoms or cells";
    default: return "unknown error code";
    }
}

int md_abi_version(void) { return MD_ABI_VERSION; }

int md_cell_dims(const double *box_L, double rc, int32_t *dims_out)
{
    if (!dims_out) return MD_ERR_INVALID_ARG;
    return compute_dims(box_L, rc, dims_out);
}

size_t md_workspace_bytes(int32_t n, const int32_t *dims)
{
    int ncell = 0;
    if (n < 0 || n > kMaxAtoms || check_dims(dims, &ncell) != MD_OK) return 0;
    return ws_layout(n, ncell, true, false, split_dims(dims)).total + kAlign;
}

int md_build_cells(const float *pos_q, const int32_t *type, int32_t n, const double *box_L,
                   const int32_t *dims, int32_t *cell_start, int32_t *perm, float *pos_q_sorted,
                   int32_t *type_sorted, void *workspace, size_t ws_bytes, uint32_t *status,
                   void *stream)
{
    int ncell = 0;
    if (n < 0 || n > kMaxAtoms) return MD_ERR_INVALID_ARG;
    int e = validate_box(box_L);
    if (e) return e;
    if ((e = check_dims(dims, &ncell))) return e;
    if (!cell_start) return MD_ERR_INVALID_ARG;
    if (n > 0 && (!pos_q || !type || !perm || !pos_q_sorted || !type_sorted)) return MD_ERR_INVALID_ARG;
    if ((pos_q && !aligned16(pos_q)) || (pos_q_sorted && !aligned16(pos_q_sorted))) return MD_ERR_INVALID_ARG;
    WsLayout ws = ws_layout(n, ncell, true, false, split_dims(dims));
    char *wsp = ws_base(workspace, ws_bytes, ws);
    if (!wsp) return MD_ERR_WORKSPACE;
    BoxF box = make_box(box_L, dims);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return cuda_code(launch_build_cells(reinterpret_cast<const float4 *>(pos_q), type, n, box,
                                        cell_start, perm, reinterpret_cast<float4 *>(pos_q_sorted),
                                        type_sorted, ws, wsp, status, s));
}

int md_nonbonded_forces_algo(const int32_t *cell_start, const int32_t *perm,
                             const float *pos_q_sorted, const int32_t *type_sorted, int32_t n,
                             const double *box_L, const int32_t *dims, const md_forcefield *ff,
                             int32_t mode, int32_t algo, void *forces_out,
                             double *energy_virial_out, unsigned long long *pair_count_out,
                             void *workspace, size_t ws_bytes, uint32_t *status, void *stream)
{
    int ncell = 0;
    if (n < 0 || n > kMaxAtoms) return MD_ERR_INVALID_ARG;
    int e = check_ff(ff);
    if (e) return e;
    if (mode != MD_ACCUM_F32 && mode != MD_ACCUM_FIXED64 && mode != MD_ACCUM_F64 &&
        mode != MD_ACCUM_FIXED_TILE)
        return MD_ERR_INVALID_ARG;
    if (algo != MD_ALGO_DEFAULT && algo != MD_ALGO_FULL_SHELL && algo != MD_ALGO_HALF_SHELL &&
        algo != MD_ALGO_CLUSTER)
        return MD_ERR_INVALID_ARG;
    if (mode == MD_ACCUM_FIXED_TILE && algo != MD_ALGO_DEFAULT && algo != MD_ALGO_CLUSTER)
        return MD_ERR_INVALID_ARG;
    int32_t want[3];
    if ((e = compute_dims(box_L, ff->rc, want))) return e;
    if ((e = check_dims(dims, &ncell))) return e;
    for (int d = 0; d < 3; ++d)
        if (dims[d] != want[d]) return MD_ERR_CUTOFF;
    if (!cell_start) return MD_ERR_INVALID_ARG;
    if (n > 0 && (!perm || !pos_q_sorted || !type_sorted || !forces_out)) return MD_ERR_INVALID_ARG;
    if (pos_q_sorted && !aligned16(pos_q_sorted)) return MD_ERR_INVALID_ARG;
    WsLayout ws = ws_layout(n, ncell, true, false, split_dims(dims));
    char *wsp = ws_base(workspace, ws_bytes, ws);
    if (!wsp) return MD_ERR_WORKSPACE;
    ForceArgs a;
    a.cell_start = cell_start;
    a.perm = perm;
    a.pos_q_sorted = reinterpret_cast<const float4 *>(pos_q_sorted);
    a.type_sorted = type_sorted;
    a.n = n;
    a.box = make_box(box_L, dims);
    a.AB = reinterpret_cast<const float2 *>(ff->AB);
    a.ntypes = ff->ntypes;
    a.k_coulomb = (float)ff->k_coulomb;
    a.k_coulomb64 = ff->k_coulomb;
    a.rc = (float)ff->rc;
    a.rc64 = ff->rc;
    a.mode = mode;
    a.algo = algo;
    a.forces_out = forces_out;
    a.energy_virial_out = energy_virial_out;
    a.pair_count_out = pair_count_out;
    a.status = status;
    return cuda_code(launch_forces(a, ws, wsp, static_cast<cudaStream_t>(stream)));
}

int md_nonbonded_forces(const int32_t *cell_start, const int32_t *perm, const float *pos_q_sorted,
                        const int32_t *type_sorted, int32_t n, const double *box_L,
                        const int32_t *dims, const md_forcefield *ff, int32_t mode,
                        void *forces_out, double *energy_virial_out,
                        unsigned long long *pair_count_out, void *workspace, size_t ws_bytes,
                        uint32_t *status, void *stream)
{
    return md_nonbonded_forces_algo(cell_start, perm, pos_q_sorted, type_sorted, n, box_L, dims, ff,
                                    mode, MD_ALGO_DEFAULT, forces_out, energy_virial_out,
                                    pair_count_out, workspace, ws_bytes, status, stream);
}

int md_step(double *pos, double *vel, void *forces, int32_t forces_valid, const float *inv_mass,
            const float *q, const int32_t *type, int32_t n, const double *box_L,
            const md_forcefield *ff, int32_t mode, double dt_fs, int32_t n_steps,
            double *energy_log, void *workspace, size_t ws_bytes, uint32_t *status, void *stream)
{
    if (n < 0 || n > kMaxAtoms || n_steps < 0) return MD_ERR_INVALID_ARG;
    if (!(dt_fs > 0.0) || !isfinite(dt_fs)) return MD_ERR_INVALID_ARG;
    int e = check_ff(ff);
    if (e) return e;
    if (mode != MD_ACCUM_F32 && mode != MD_ACCUM_FIXED64 && mode != MD_ACCUM_F64 &&
        mode != MD_ACCUM_FIXED_TILE)
        return MD_ERR_INVALID_ARG;
    int32_t dims[3];
    if ((e = compute_dims(box_L, ff->rc, dims))) return e;
    if (n > 0 && (!pos || !vel || !forces || !inv_mass || !q || !type)) return MD_ERR_INVALID_ARG;
    int ncell = dims[0] * dims[1] * dims[2];
    WsLayout ws = ws_layout(n, ncell, true, false, split_dims(dims));
    char *wsp = ws_base(workspace, ws_bytes, ws);
    if (!wsp) return MD_ERR_WORKSPACE;
    if (n == 0 || (n_steps == 0 && forces_valid)) return MD_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BoxF box = make_box(box_L, dims);
    int32_t *cs = reinterpret_cast<int32_t *>(wsp + ws.st_cell_start);
    int32_t *pm = reinterpret_cast<int32_t *>(wsp + ws.st_perm);
    float4 *pqs = reinterpret_cast<float4 *>(wsp + ws.st_pos_q_sorted);
    int32_t *tys = reinterpret_cast<int32_t *>(wsp + ws.st_type_sorted);
    float4 *pq = reinterpret_cast<float4 *>(wsp + ws.st_pos_q);
    double *ev = reinterpret_cast<double *>(wsp + ws.ev);

    ForceArgs a;
    a.cell_start = cs;
    a.perm = pm;
    a.pos_q_sorted = pqs;
    a.type_sorted = tys;
    a.n = n;
    a.box = box;
    a.AB = reinterpret_cast<const float2 *>(ff->AB);
    a.ntypes = ff->ntypes;
    a.k_coulomb = (float)ff->k_coulomb;
    a.k_coulomb64 = ff->k_coulomb;
    a.rc = (float)ff->rc;
    a.rc64 = ff->rc;
    a.mode = mode;
    a.algo = MD_ALGO_DEFAULT;
    a.forces_out = forces;
    a.pair_count_out = nullptr;
    a.status = status;

    cudaError_t ce;
    const double half_dt = 0.5 * dt_fs;
    // the step's passes fused: [half kick +] drift + wrap + cell build in cluster order,
    // then the forces with the second half kick in their last pass
    a.presorted = 1;
    a.accum_zeroed = mode != MD_ACCUM_F64;  // the build pass zeroes the accumulators
    a.clu_box = reinterpret_cast<const float4 *>(wsp + ws.clu_box);  // written by the build
    a.kick_inv_mass = inv_mass;
    a.kick_half_dt = half_dt;
    auto build = [&](bool kick, double dt) -> cudaError_t {
        return launch_kick_drift_build(pos, vel, forces, mode, inv_mass, q, type, n, box, nullptr, dt,
                                       half_dt, kick, pq, cs, pm, pqs, tys, ws, wsp, status, s);
    };
    auto eval_forces = [&](bool energy, bool kick) -> cudaError_t {
        a.energy_virial_out = energy ? ev : nullptr;
        a.kick_vel = kick ? vel : nullptr;
        return launch_forces(a, ws, wsp, s);
    };
    if (!forces_valid) {
        // wrap the start positions and make the float copy, then F(x0)
        if ((ce = build(false, 0.0)) != cudaSuccess) return MD_ERR_CUDA;
        if ((ce = eval_forces(false, false)) != cudaSuccess) return MD_ERR_CUDA;
    }
    for (int st = 0; st < n_steps; ++st) {
        if ((ce = build(true, dt_fs)) != cudaSuccess) return MD_ERR_CUDA;
        if ((ce = eval_forces(energy_log != nullptr, true)) != cudaSuccess) return MD_ERR_CUDA;
        if (energy_log) {
            ce = launch_energy_log_row(vel, inv_mass, n, ev, energy_log + 4 * (size_t)st, ws, wsp, s);
            if (ce != cudaSuccess) return MD_ERR_CUDA;
        }
    }
    return MD_OK;
}

size_t md_verlet_workspace_bytes(int32_t n, const double *box_L, double rc, double skin)
{
    int32_t dims[3];
    if (n < 0 || n > kMaxAtoms || !(skin > 0.0) || !isfinite(skin)) return 0;
    if (compute_dims(box_L, rc + skin, dims) != MD_OK) return 0;
    return ws_layout(n, dims[0] * dims[1] * dims[2], false, true, split_dims(dims)).total + kAlign;
}

int md_step_verlet(double *pos, double *vel, void *forces, int32_t forces_valid,
                   const float *inv_mass, const float *q, const int32_t *type, int32_t n,
                   const double *box_L, const md_forcefield *ff, int32_t mode, double dt_fs,
                   int32_t n_steps, double skin, double *energy_log,
                   unsigned long long *rebuilds, void *workspace, size_t ws_bytes,
                   uint32_t *status, void *stream)
{
    if (n < 0 || n > kMaxAtoms || n_steps < 0) return MD_ERR_INVALID_ARG;
    if (!(dt_fs > 0.0) || !isfinite(dt_fs)) return MD_ERR_INVALID_ARG;
    if (!(skin > 0.0) || !isfinite(skin)) return MD_ERR_INVALID_ARG;
    int e = check_ff(ff);
    if (e) return e;
    if (mode != MD_ACCUM_F32 && mode != MD_ACCUM_FIXED64 && mode != MD_ACCUM_FIXED_TILE)
        return MD_ERR_INVALID_ARG;
    int32_t dims[3];
    if ((e = compute_dims(box_L, ff->rc, dims))) return e;       // rc itself
    if ((e = compute_dims(box_L, ff->rc + skin, dims))) return e;  // the Verlet grid
    if (n > 0 && (!pos || !vel || !forces || !inv_mass || !q || !type)) return MD_ERR_INVALID_ARG;
    const int ncell = dims[0] * dims[1] * dims[2];
    WsLayout ws = ws_layout(n, ncell, false, true, split_dims(dims));
    char *wsp = ws_base(workspace, ws_bytes, ws);
    if (!wsp) return MD_ERR_WORKSPACE;
    if (n == 0 || (n_steps == 0 && forces_valid)) return MD_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BoxF box = make_box(box_L, dims);
    int32_t *cs = reinterpret_cast<int32_t *>(wsp + ws.st_cell_start);
    int32_t *pm = reinterpret_cast<int32_t *>(wsp + ws.st_perm);
    float4 *pqs = reinterpret_cast<float4 *>(wsp + ws.st_pos_q_sorted);
    int32_t *tys = reinterpret_cast<int32_t *>(wsp + ws.st_type_sorted);
    float4 *pq = reinterpret_cast<float4 *>(wsp + ws.st_pos_q);
    float4 *x_ref = reinterpret_cast<float4 *>(wsp + ws.v_ref);
    VerletFlags *flags = reinterpret_cast<VerletFlags *>(wsp + ws.v_flags);
    double *ev = reinterpret_cast<double *>(wsp + ws.ev);
    void *accum = wsp + ws.accum;
    // rebuild when an atom has moved s/2 or more since the cells were built (less a
    // margin for the float rounding of the positions the move is measured on)
    const double lmax = fmax(box_L[0], fmax(box_L[1], box_L[2]));
    const double half_skin = 0.5 * skin - 4.0 * 1.1920929e-7 * lmax;  // a few float ulps of L
    const float threshold2 = half_skin > 0.0 ? (float)(half_skin * half_skin) : 0.0f;

    ForceArgs a;
    a.cell_start = cs;
    a.perm = pm;
    a.pos_q_sorted = pqs;
    a.type_sorted = tys;
    a.n = n;
    a.box = box;
    a.AB = reinterpret_cast<const float2 *>(ff->AB);
    a.ntypes = ff->ntypes;
    a.k_coulomb = (float)ff->k_coulomb;
    a.k_coulomb64 = ff->k_coulomb;
    a.rc = (float)ff->rc;
    a.rc64 = ff->rc;
    a.mode = mode;
    a.algo = MD_ALGO_CLUSTER;
    a.forces_out = forces;
    a.pair_count_out = nullptr;
    a.status = status;
    a.presorted = 1;
    a.accum_zeroed = 1;  // the drift pass zeroes the accumulators
    a.gather_pq = pq;
    a.kick_inv_mass = inv_mass;
    const double half_dt = 0.5 * dt_fs;
    a.kick_half_dt = half_dt;
    const int *run = &flags->rebuild;
    // every step's passes: [half kick +] drift + wrap + float copy + largest move, the
    // rebuild decision, the rebuild kernels (which return at once without one), the forces
    // through the kept cells and the second half kick; the first step of a call rebuilds
    auto step = [&](bool kick, double dt, bool first, bool energy, bool kick2) -> cudaError_t {
        cudaError_t ce = launch_verlet_drift(pos, vel, forces, mode, inv_mass, q, n, box, dt, half_dt,
                                             kick, pq, x_ref, accum, flags, status, s);
        if (ce == cudaSuccess) ce = launch_verlet_decide(flags, threshold2, first, rebuilds, s);
        if (ce == cudaSuccess)
            ce = launch_verlet_rebuild(pq, type, n, box, cs, pm, pqs, tys, x_ref, run, ws, wsp, status, s);
        if (ce != cudaSuccess) return ce;
        a.energy_virial_out = energy ? ev : nullptr;
        a.kick_vel = kick2 ? vel : nullptr;
        return launch_forces(a, ws, wsp, s);
    };
    bool first = true;
    if (!forces_valid) {
        if (step(false, 0.0, true, false, false) != cudaSuccess) return MD_ERR_CUDA;
        first = false;
    }
    for (int st = 0; st < n_steps; ++st) {
        if (step(true, dt_fs, first, energy_log != nullptr, true) != cudaSuccess) return MD_ERR_CUDA;
        first = false;
        if (energy_log) {
            cudaError_t ce = launch_energy_log_row(vel, inv_mass, n, ev, energy_log + 4 * (size_t)st, ws, wsp, s);
            if (ce != cudaSuccess) return MD_ERR_CUDA;
        }
    }
    return MD_OK;
}

size_t md_batch_workspace_bytes(int32_t nsys, const md_system_desc *systems)
{
    BatchLayout bl;
    std::vector<int32_t> dims;
    if (batch_layout(nsys, systems, &bl, &dims) != MD_OK) return 0;
    return bl.total + kAlign;
}

// The batch's descriptor block (per-system SysDesc, cell -> system, the cell list of each
// regime, atom -> system) filled into `host` with the device layout of bytes
// [0, bl.run_base) of the batch workspace.
static void fill_batch_block(int32_t nsys, const md_system_desc *systems, const BatchLayout &bl,
                             const std::vector<int32_t> &dims, char *host)
{
    SysDesc *sys = reinterpret_cast<SysDesc *>(host + bl.sys);
    int *cell_sys = reinterpret_cast<int *>(host + bl.cell_sys);
    int *cell_list = reinterpret_cast<int *>(host + bl.cell_list);
    int *atom_sys = reinterpret_cast<int *>(host + bl.atom_sys);
    int atom = 0, cell = 0, reg = 0, mi = bl.ncell_reg;
    for (int s = 0; s < nsys; ++s) {
        const md_system_desc &d = systems[s];
        SysDesc o;
        memset(&o, 0, sizeof(o));
        o.box = make_box(d.box_L, dims.data() + 3 * s);
        o.AB = reinterpret_cast<const float2 *>(d.ff.AB);
        o.ntypes = d.ff.ntypes;
        o.kc = (float)d.ff.k_coulomb;
        o.kc64 = d.ff.k_coulomb;
        o.mi = half_shell_pairs_per_cell(o.box) == 27;
        cutoff_thresholds(o.box, d.ff.rc, o.mi != 0, &o.rc2, &o.rc2m);
        o.atom_offset = atom;
        o.natoms = d.n;
        o.cell_offset = cell;
        memcpy(&sys[s], &o, sizeof(o));
        for (int c = 0; c < o.box.ncell; ++c) {
            cell_sys[(size_t)cell + c] = s;
            cell_list[(size_t)(o.mi ? mi++ : reg++)] = cell + c;
        }
        for (int i = 0; i < d.n; ++i) atom_sys[(size_t)atom + i] = s;
        atom += d.n;
        cell += o.box.ncell;
    }
}

int md_batch_prepare(int32_t nsys, const md_system_desc *systems, void *workspace, size_t ws_bytes,
                     void *stream)
{
    BatchLayout bl;
    std::vector<int32_t> dims;
    int e = batch_layout(nsys, systems, &bl, &dims);
    if (e) return e;
    if (!workspace) return MD_ERR_WORKSPACE;
    uintptr_t p = reinterpret_cast<uintptr_t>(workspace);
    uintptr_t a = (p + kAlign - 1) & ~(uintptr_t)(kAlign - 1);
    if (ws_bytes < (a - p) + bl.total) return MD_ERR_WORKSPACE;
    char *wsp = reinterpret_cast<char *>(a);
    std::vector<char> host(bl.run_base);
    fill_batch_block(nsys, systems, bl, dims, host.data());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t ce = cudaMemcpyAsync(wsp, host.data(), bl.run_base, cudaMemcpyHostToDevice, st);
    // the host vector is released on return: wait for the copy to finish reading it
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    return ce == cudaSuccess ? MD_OK : MD_ERR_CUDA;
}

size_t md_batch_staging_bytes(int32_t nsys, const md_system_desc *systems)
{
    BatchLayout bl;
    std::vector<int32_t> dims;
    if (batch_layout(nsys, systems, &bl, &dims) != MD_OK) return 0;
    return bl.run_base;
}

int md_batch_prepare_staged(int32_t nsys, const md_system_desc *systems, void *workspace,
                            size_t ws_bytes, void *host_staging, size_t staging_bytes,
                            void *stream)
{
    BatchLayout bl;
    std::vector<int32_t> dims;
    int e = batch_layout(nsys, systems, &bl, &dims);
    if (e) return e;
    if (!workspace) return MD_ERR_WORKSPACE;
    uintptr_t p = reinterpret_cast<uintptr_t>(workspace);
    uintptr_t a = (p + kAlign - 1) & ~(uintptr_t)(kAlign - 1);
    if (ws_bytes < (a - p) + bl.total) return MD_ERR_WORKSPACE;
    if (!host_staging || staging_bytes < bl.run_base) return MD_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(host_staging) & 15u) return MD_ERR_INVALID_ARG;
    char *wsp = reinterpret_cast<char *>(a);
    fill_batch_block(nsys, systems, bl, dims, static_cast<char *>(host_staging));
    cudaError_t ce = cudaMemcpyAsync(wsp, host_staging, bl.run_base, cudaMemcpyHostToDevice,
                                     static_cast<cudaStream_t>(stream));
    return ce == cudaSuccess ? MD_OK : MD_ERR_CUDA;
}

int md_batch_step(int32_t nsys, const md_system_desc *systems, double *pos, double *vel,
                  void *forces, int32_t forces_valid, const float *inv_mass, const float *q,
                  const int32_t *type, int32_t mode, double dt_fs, int32_t n_steps,
                  unsigned long long *pair_count, void *workspace, size_t ws_bytes,
                  uint32_t *status, void *stream)
{
    return md_batch_step_tuned(nsys, systems, pos, vel, forces, forces_valid, inv_mass, q, type,
                               mode, dt_fs, n_steps, pair_count, workspace, ws_bytes, status,
                               nullptr, stream);
}

int md_batch_step_tuned(int32_t nsys, const md_system_desc *systems, double *pos, double *vel,
                        void *forces, int32_t forces_valid, const float *inv_mass,
                        const float *q, const int32_t *type, int32_t mode, double dt_fs,
                        int32_t n_steps, unsigned long long *pair_count, void *workspace,
                        size_t ws_bytes, uint32_t *status, const md_batch_tuning *tuning,
                        void *stream)
{
    const int shape_reg = tuning ? tuning->shape_regular : 0;
    const int shape_mi = tuning ? tuning->shape_small : 0;
    if (shape_reg < 0 || shape_reg >= MD_BATCH_SHAPES || shape_mi < 0 || shape_mi >= MD_BATCH_SHAPES)
        return MD_ERR_INVALID_ARG;
    BatchLayout bl;
    std::vector<int32_t> dims;
    int e = batch_layout(nsys, systems, &bl, &dims);
    if (e) return e;
    if (n_steps < 0 || !(dt_fs > 0.0) || !isfinite(dt_fs)) return MD_ERR_INVALID_ARG;
    if (mode != MD_ACCUM_F32 && mode != MD_ACCUM_FIXED64 && mode != MD_ACCUM_FIXED_TILE)
        return MD_ERR_INVALID_ARG;
    // MD_ACCUM_FIXED_TILE runs on the cluster kernel only: shapes 0 and 5
    if (mode == MD_ACCUM_FIXED_TILE &&
        ((shape_reg != 0 && shape_reg != 5) || (shape_mi != 0 && shape_mi != 5)))
        return MD_ERR_INVALID_ARG;
    if (bl.n > 0 && (!pos || !vel || !forces || !inv_mass || !q || !type)) return MD_ERR_INVALID_ARG;
    if (!workspace) return MD_ERR_WORKSPACE;
    uintptr_t p = reinterpret_cast<uintptr_t>(workspace);
    uintptr_t al = (p + kAlign - 1) & ~(uintptr_t)(kAlign - 1);
    if (ws_bytes < (al - p) + bl.total) return MD_ERR_WORKSPACE;
    char *wsp = reinterpret_cast<char *>(al);
    if (bl.n == 0 || (n_steps == 0 && forces_valid)) return MD_OK;
    BatchArgs b;
    b.sys = reinterpret_cast<const SysDesc *>(wsp + bl.sys);
    b.cell_sys = reinterpret_cast<const int *>(wsp + bl.cell_sys);
    b.cell_list = reinterpret_cast<const int *>(wsp + bl.cell_list);
    b.atom_sys = reinterpret_cast<const int *>(wsp + bl.atom_sys);
    b.nsys = bl.nsys;
    b.n = bl.n;
    b.ncell = bl.ncell;
    b.ncell_mi = bl.ncell_mi;
    b.ncell_reg = bl.ncell_reg;
    b.max_ntypes = 0;
    for (int k = 0; k < nsys; ++k) b.max_ntypes = systems[k].ff.ntypes > b.max_ntypes ? systems[k].ff.ntypes : b.max_ntypes;
    char *run = wsp + bl.run_base;
    const WsLayout &ws = bl.run;
    int32_t *cs = reinterpret_cast<int32_t *>(run + ws.st_cell_start);
    int32_t *pm = reinterpret_cast<int32_t *>(run + ws.st_perm);
    float4 *pqs = reinterpret_cast<float4 *>(run + ws.st_pos_q_sorted);
    int32_t *tys = reinterpret_cast<int32_t *>(run + ws.st_type_sorted);
    float4 *pq = reinterpret_cast<float4 *>(run + ws.st_pos_q);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double half_dt = 0.5 * dt_fs;
    ForceArgs a = {};
    a.cell_start = cs;
    a.perm = pm;
    a.pos_q_sorted = pqs;
    a.type_sorted = tys;
    a.n = bl.n;
    a.mode = mode;
    a.forces_out = forces;
    a.status = status;
    // the same fused passes as md_step, over the whole batch
    a.presorted = 1;
    a.accum_zeroed = mode != MD_ACCUM_F64;  // the build pass zeroes the accumulators
    a.kick_inv_mass = inv_mass;
    a.kick_half_dt = half_dt;
    auto build = [&](bool kick, double dt) -> cudaError_t {
        return launch_kick_drift_build(pos, vel, forces, mode, inv_mass, q, type, bl.n, BoxF{}, &b, dt,
                                       half_dt, kick, pq, cs, pm, pqs, tys, ws, run, status, s);
    };
    auto eval_forces = [&](bool kick) -> cudaError_t {
        a.kick_vel = kick ? vel : nullptr;
        return launch_forces_batched(a, b, pair_count, ws, run, s, shape_reg, shape_mi);
    };
    if (!forces_valid) {
        if (build(false, 0.0) != cudaSuccess) return MD_ERR_CUDA;
        if (eval_forces(false) != cudaSuccess) return MD_ERR_CUDA;
    }
    for (int st = 0; st < n_steps; ++st) {
        if (build(true, dt_fs) != cudaSuccess) return MD_ERR_CUDA;
        if (eval_forces(true) != cudaSuccess) return MD_ERR_CUDA;
    }
    return MD_OK;
}

}  // extern "C"
