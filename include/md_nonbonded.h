/*
 * md_nonbonded.h -- C ABI of the GB300 cutoff non-bonded molecular-dynamics force path.
 *
 * The library evaluates the short-range non-bonded forces of the paper
 * (Section II.A): Lennard-Jones, Eq. 1  F = (A/|r|^14 - B/|r|^8) * r, plus
 * Coulomb, Eq. 2  F = k*q1*q2/|r|^3 * r, for every pair of atoms closer than
 * the cutoff radius rc (strictly: r^2 < rc^2), found through a periodic cell
 * list whose cells have edge >= rc, so that each home cell meets only its
 * 3x3x3 neighbour cells (Section II.A, Fig. 2, Algorithm 1).  Beyond rc the
 * force is zero; long-range electrostatics is outside this library (the paper
 * leaves it to the host).  A velocity-Verlet integrator wraps the force call.
 *
 * Conventions shared by every entry point
 *   - Units: Angstrom, fs, amu, elementary charge, kcal/mol.
 *   - r = x_i - x_j under the minimum-image convention; the force above acts
 *     on atom i and its reaction -F on atom j.
 *   - All array arguments are DEVICE pointers owned by the caller unless the
 *     comment says "host".  The library never allocates, frees or keeps caller
 *     memory; scratch lives in the caller's `workspace` (size from
 *     md_workspace_bytes).  Every call is asynchronous on `stream` (a
 *     cudaStream_t passed as void*; NULL is the legacy default stream) and
 *     returns after enqueuing its kernels.
 *   - Return value: MD_OK (0) or a negative MD_ERR_* code from host-side
 *     validation or a failed launch; nothing is enqueued when validation fails.
 *   - Conditions found on the device are OR-ed into *status (a device uint32
 *     the caller zeroes and reads after synchronising; may be NULL) as
 *     MD_STATUS_* bits.  Kernels never trap.
 *   - Box: host double[3] edge lengths of an orthorhombic periodic box.  The
 *     cutoff must satisfy 0 < rc < min(L)/2 (else MD_ERR_CUTOFF).
 *   - Cells: dims[d] = max(1, floor(L_d / rc)) per axis (md_cell_dims); a
 *     coordinate x is wrapped in FP64 as w = x - L*floor(x/L) folded into
 *     [0, L), its cell index along the axis is floor(w * (dims/L)) clamped to
 *     [0, dims-1], the flat cell index is cx + dims0*(cy + dims1*cz), and the
 *     atoms of a cell are kept in ascending input order.
 */
#ifndef MD_NONBONDED_H
#define MD_NONBONDED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MD_ABI_VERSION 1

/* return codes */
#define MD_OK 0
#define MD_ERR_INVALID_ARG (-1) /* n < 0, NULL where required, ntypes outside 1..32, dt <= 0 ... */
#define MD_ERR_CUTOFF (-2)      /* rc <= 0, rc >= min(L)/2, or dims disagree with md_cell_dims */
#define MD_ERR_WORKSPACE (-3)   /* workspace NULL or smaller than md_workspace_bytes */
#define MD_ERR_CUDA (-4)        /* a kernel launch or async CUDA call failed */
#define MD_ERR_TOO_LARGE (-5)   /* more cells or atoms than the index types hold */

/* device status bits */
#define MD_STATUS_NONFINITE 1u      /* a non-finite position or force was seen */
#define MD_STATUS_FIXED_OVERFLOW 2u /* a term reached 2^31 kcal/mol/A in a fixed-point mode */
#define MD_STATUS_BAD_TYPE 4u       /* an LJ type outside [0, ntypes) was read as type 0 */

/* accumulation / precision modes (argument `mode`) */
#define MD_ACCUM_F32 0     /* FP32 pair math and FP32 accumulation; forces float[n][3] */
#define MD_ACCUM_FIXED64 1 /* FP32 pair math; every pair term rounded (to nearest even) to a
                              two's-complement int64 at scale 2^32 and summed exactly, so the
                              result is independent of summation order and bit-reproducible;
                              forces int64[n][3] (divide by 2^32 for kcal/mol/A) */
#define MD_ACCUM_F64 2     /* FP64 pair math and accumulation, a slow reference mode;
                              forces double[n][3] */
#define MD_ACCUM_FIXED_TILE 3 /* FP32 pair math and FP32 partial sums, each partial rounded
                              once to the int64 grid of MD_ACCUM_FIXED64 and summed exactly:
                              a home cluster's sums per neighbour tile, and a neighbour
                              tile's reactions.  The partials are formed in a fixed order
                              (no floating-point atomics), so results are bit-reproducible
                              run to run for the same inputs, but they depend on the cell
                              and cluster order and differ from MD_ACCUM_FIXED64's bits;
                              forces int64[n][3] as in MD_ACCUM_FIXED64.  Cluster kernel only
                              (MD_ALGO_DEFAULT or MD_ALGO_CLUSTER; batch shapes 0 and 5) */

/* force-kernel choice for md_nonbonded_forces_algo.  MD_ALGO_DEFAULT (what
 * md_nonbonded_forces and md_step use): MD_ALGO_CLUSTER for MD_ACCUM_F32 and
 * MD_ACCUM_FIXED64, MD_ALGO_FULL_SHELL for MD_ACCUM_F64 (its only kernel). */
#define MD_ALGO_DEFAULT 0 /* MD_ACCUM_FIXED_TILE: MD_ALGO_CLUSTER */
#define MD_ALGO_FULL_SHELL 1 /* one thread per home atom over all 27 neighbour cells (Alg. 1) */
#define MD_ALGO_HALF_SHELL 2 /* each cell pair once, reactions by Newton's third law */
#define MD_ALGO_CLUSTER 3    /* the half shell filtered by clusters of 8 atoms, every pair of
                                a cluster pair in range evaluated (per-pair minimum image in
                                boxes with an axis of 2 cells).  MD_ACCUM_F32 without
                                energies, on grids large enough to fill the GPU: each home
                                cluster against all its in-range neighbour clusters of a
                                group of cells at once; otherwise one cluster pair per warp
                                step.  The two give the same forces up to FP32 rounding. */

/* Force-field constants of Eq. 1-2.  Host struct; AB is a DEVICE pointer to
 * float[ntypes][ntypes][2] holding (A_ij, B_ij) of Eq. 1 (symmetric in i,j). */
typedef struct md_forcefield {
    int32_t ntypes;   /* 1..32 */
    int32_t reserved; /* set to 0 */
    const float *AB;
    double k_coulomb; /* k of Eq. 2, kcal*A/(mol*e^2), e.g. 332.0636 */
    double rc;        /* cutoff radius, A */
} md_forcefield;

/* Human-readable text for a return code (static storage, never NULL). */
const char *md_strerror(int code);

/* MD_ABI_VERSION of the loaded library. */
int md_abi_version(void);

/* Cells per axis for a box and cutoff (Section II.A: cell edge roughly equal to rc,
 * here edge >= rc).  Host only: box_L host double[3], dims_out host int32[3].
 * MD_ERR_CUTOFF when rc <= 0 or rc >= min(L)/2. */
int md_cell_dims(const double *box_L, double rc, int32_t *dims_out);

/* Bytes of scratch every entry point below needs for n atoms and these cell dims
 * (host int32[3]); 0 on invalid arguments.  One workspace of this size serves
 * any entry point, but concurrent calls must not share one. */
size_t md_workspace_bytes(int32_t n, const int32_t *dims);

/*
 * md_build_cells -- bin atoms into cells by a counting sort (Section II.A cell list;
 * Section II.B item 2: per-cell arrays instead of linked lists).
 *   pos_q         [n][4] float: x, y, z, q in input order (any real coordinates;
 *                 they are wrapped into the box)
 *   type          [n] int32 LJ type
 *   dims          host int32[3] from md_cell_dims(box_L, rc)
 * Outputs (device, caller-allocated):
 *   cell_start    [ncell+1] int32: atoms of cell c are sorted slots
 *                 cell_start[c] .. cell_start[c+1]-1, ncell = dims0*dims1*dims2
 *   perm          [n] int32: sorted slot -> input index
 *   pos_q_sorted  [n][4] float: wrapped x, y, z (rounded to float from the FP64
 *                 wrap) and q, in sorted order
 *   type_sorted   [n] int32, in sorted order
 * A non-finite coordinate sets MD_STATUS_NONFINITE and the atom goes to cell 0 at
 * the origin.  The result is deterministic (stable order within a cell).
 */
int md_build_cells(const float *pos_q, const int32_t *type, int32_t n, const double *box_L,
                   const int32_t *dims, int32_t *cell_start, int32_t *perm, float *pos_q_sorted,
                   int32_t *type_sorted, void *workspace, size_t ws_bytes, uint32_t *status,
                   void *stream);

/*
 * md_build_cells_noalloc -- md_build_cells for callers that cannot allocate device memory
 * (no counterpart in the paper; a convenience of this library).
 *
 * Some callers cannot call cudaMalloc, or any routine that allocates, at the point where
 * they bin atoms: a plugin handed only its input and output buffers by a host program,
 * code running while other work on the device is being recorded, or an application
 * whose allocator forbids new allocations inside its step.  This variant takes no
 * workspace: its scratch lives in one fixed-size device array inside the library, so
 * the call allocates nothing.  Inputs, outputs, their layouts and the result are those
 * of md_build_cells (the outputs are bit-identical).
 *   Limits: n <= MD_NOALLOC_MAX_ATOMS and dims0*dims1*dims2 <= MD_NOALLOC_MAX_CELLS,
 *   else MD_ERR_TOO_LARGE and nothing is enqueued.  Every GPU that loads the library
 *   holds MD_NOALLOC_SCRATCH_BYTES for this array until the process exits.
 *   The first call on each device looks up the array's device address on that device
 *   (the current one) and keeps it for the life of the process; make that first call
 *   before any stream capture begins.  The kept address is not valid after the device is
 *   reset (cudaDeviceReset, or a runtime that tears down the primary context): the module
 *   is loaded again and may land elsewhere, so do not call this entry point after such
 *   a reset in the same process.
 *   All calls on a device share the array and it keeps the last call's contents (the
 *   counters are cleared on every call).  Calls that overlap on the GPU race on it and
 *   give wrong cell lists: issue them in order on one stream.
 */
#define MD_NOALLOC_MAX_ATOMS 131072
#define MD_NOALLOC_MAX_CELLS 16384
#define MD_NOALLOC_SCRATCH_BYTES 1114112 /* 2 x 4 B x MAX_ATOMS + 4 B x MAX_CELLS */
int md_build_cells_noalloc(const float *pos_q, const int32_t *type, int32_t n,
                           const double *box_L, const int32_t *dims, int32_t *cell_start,
                           int32_t *perm, float *pos_q_sorted, int32_t *type_sorted,
                           uint32_t *status, void *stream);

/*
 * md_nonbonded_forces -- short-range non-bonded forces (Eq. 1 + Eq. 2 with the cutoff of
 * Section II.A) over the cell list that md_build_cells produced, in the order of
 * Algorithm 1: each home cell meets its neighbour cells, each candidate pair passes
 * the filter r^2 < rc^2, and only the surviving pairs reach the force computation.
 *   cell_start, perm, pos_q_sorted, type_sorted   as returned by md_build_cells
 *   ff            host pointer to the force field (AB on the device)
 *   mode          MD_ACCUM_F32 / MD_ACCUM_FIXED64 / MD_ACCUM_F64 / MD_ACCUM_FIXED_TILE
 *   forces_out    [n][3] in INPUT atom order; element type by mode (float, int64,
 *                 double, int64); fully overwritten (the callee zeroes it)
 *   energy_virial_out  device double[3] = {E_LJ, E_Coulomb, W} or NULL, with
 *                 U_LJ = A/(12 r^12) - B/(6 r^6), U_C = k q1 q2 / r, W = sum f r^2
 *                 (F = f r); summed per block and then in a fixed order
 *   pair_count_out     device uint64[1] or NULL: unique pairs with r^2 < rc^2
 * Forces and counts of modes FIXED64, F64 and FIXED_TILE are reproducible bit for bit;
 * F32 adds partial sums (per home cluster and row or tile, per neighbour atom and step or
 * tile) with floating-point atomics and may differ in the last bits between runs.  MD_ERR_INVALID_ARG for MD_ACCUM_FIXED_TILE
 * with MD_ALGO_FULL_SHELL or MD_ALGO_HALF_SHELL.
 */
int md_nonbonded_forces(const int32_t *cell_start, const int32_t *perm, const float *pos_q_sorted,
                        const int32_t *type_sorted, int32_t n, const double *box_L,
                        const int32_t *dims, const md_forcefield *ff, int32_t mode,
                        void *forces_out, double *energy_virial_out,
                        unsigned long long *pair_count_out, void *workspace, size_t ws_bytes,
                        uint32_t *status, void *stream);

/* The same with an explicit force kernel (MD_ALGO_*).  Every algorithm computes the
 * same forces up to floating-point rounding (bit for bit in FIXED64 and F64). */
int md_nonbonded_forces_algo(const int32_t *cell_start, const int32_t *perm,
                             const float *pos_q_sorted, const int32_t *type_sorted, int32_t n,
                             const double *box_L, const int32_t *dims, const md_forcefield *ff,
                             int32_t mode, int32_t algo, void *forces_out,
                             double *energy_virial_out, unsigned long long *pair_count_out,
                             void *workspace, size_t ws_bytes, uint32_t *status, void *stream);

/*
 * md_step -- n_steps of kick-drift-kick velocity Verlet around the force call (the
 * paper's iteration: forces, then the motion update; Sections I and II.A).  Per step:
 *   v += dt/2 * a;  x += dt * v;  x <- wrap(x);  rebuild cells;  F = F(x);  v += dt/2 * a
 * with a = F * inv_mass * 4.184e-4 (A/fs^2 per (kcal/mol/A)/amu).  Positions and
 * velocities are FP64 state; the force call sees the positions rounded to float.
 *   pos           [n][3] double in/out, A (wrapped into the box on exit)
 *   vel           [n][3] double in/out, A/fs
 *   forces        [n][3] in/out in the mode's element type: on entry F(pos) when
 *                 forces_valid != 0 (else it is computed first), on exit F(pos_out)
 *   inv_mass      [n] float, 1/amu;  q [n] float;  type [n] int32
 *   energy_log    device double[n_steps][4] = {E_LJ, E_Coulomb, KE, W} after each
 *                 step, or NULL (then no energies are computed)
 * The cells are rebuilt every step (no Verlet skin).  Status bits as above.
 */
int md_step(double *pos, double *vel, void *forces, int32_t forces_valid, const float *inv_mass,
            const float *q, const int32_t *type, int32_t n, const double *box_L,
            const md_forcefield *ff, int32_t mode, double dt_fs, int32_t n_steps,
            double *energy_log, void *workspace, size_t ws_bytes, uint32_t *status,
            void *stream);

/*
 * md_step_verlet -- md_step with a Verlet skin: the cells are built with edge >= rc + skin
 * and kept, with the order of the atoms within them, while no atom has moved skin/2 or
 * more since they were built; then they are built again (Section II.A's cell method,
 * reused across steps).  Every pair closer than rc lies in neighbouring kept cells, so the
 * forces are those of md_step: in MD_ACCUM_FIXED64 the same bits, step for step, and in
 * MD_ACCUM_F32 the same up to the order of summation.  The force kernel reads the current
 * positions through the kept order and filters cluster pairs on their current boxes; an
 * atom that crosses a face of the box while the cells are kept is handled by the
 * per-pair minimum image.  The rebuild decision is taken on the device (no host
 * synchronisation): each step measures the largest move since the last build, and the
 * rebuild kernels return at once when none is needed.
 *   skin          A, > 0, with rc + skin < min(L)/2 (else MD_ERR_CUTOFF)
 *   mode          MD_ACCUM_F32, MD_ACCUM_FIXED64 or MD_ACCUM_FIXED_TILE
 *   rebuilds      device uint64[1] or NULL: the number of cell builds is added to it
 *   workspace     md_verlet_workspace_bytes(n, box_L, ff->rc, skin) bytes.  The kept
 *                 cells live in it only for the duration of one call: the first step of
 *                 every call builds them.
 * Other arguments, outputs and status bits as md_step.
 */
size_t md_verlet_workspace_bytes(int32_t n, const double *box_L, double rc, double skin);
int md_step_verlet(double *pos, double *vel, void *forces, int32_t forces_valid,
                   const float *inv_mass, const float *q, const int32_t *type, int32_t n,
                   const double *box_L, const md_forcefield *ff, int32_t mode, double dt_fs,
                   int32_t n_steps, double skin, double *energy_log,
                   unsigned long long *rebuilds, void *workspace, size_t ws_bytes,
                   uint32_t *status, void *stream);

/*
 * Batches of independent systems (many small MD problems advanced together; the
 * paper's method applied to each system independently).
 *
 * The systems are stored back to back: system s owns atoms off[s] .. off[s+1]-1 of
 * every per-atom array, off[0] = 0, off[s+1] = off[s] + systems[s].n.  Each system has
 * its own box, cutoff and force field and obeys the rules of md_cell_dims.  Cells of
 * all systems are numbered globally and each launch covers every system: one kernel
 * grid for the systems with >= 3 cells per axis, one for those with an axis of 2.
 */
typedef struct md_system_desc {
    int32_t n;        /* atoms of this system */
    int32_t reserved; /* set to 0 */
    double box_L[3];
    md_forcefield ff; /* ff.AB is a DEVICE pointer; may be shared between systems */
} md_system_desc;

/* Workspace bytes for a batch (0 on invalid systems). */
size_t md_batch_workspace_bytes(int32_t nsys, const md_system_desc *systems);

/* Writes the batch's per-system descriptors into the workspace (host -> device copies,
 * then waits for them).  Call once per batch before md_batch_step, and again whenever
 * the systems change; the workspace must stay with this batch. */
int md_batch_prepare(int32_t nsys, const md_system_desc *systems, void *workspace,
                     size_t ws_bytes, void *stream);

/* md_batch_prepare without waiting on the host.  md_batch_prepare copies the descriptors
 * from memory it owns only for the duration of the call, so it waits for the stream to
 * finish the copy (and everything enqueued before it).  A caller that keeps work queued
 * on the stream while it rebuilds a batch (a server adding and removing systems between
 * steps) passes a staging buffer instead:
 *   host_staging  HOST memory of at least md_batch_staging_bytes(nsys, systems) bytes,
 *                 16-byte aligned, owned by the caller; page-locked (cudaHostAlloc or an
 *                 equivalent) so that the copy runs asynchronously.  The call writes the
 *                 descriptors into it and enqueues one copy to the device on `stream`; the
 *                 caller must not modify or free the buffer until that copy has completed
 *                 (for example, until an event recorded on `stream` after the call has
 *                 completed).
 * Errors as md_batch_prepare; MD_ERR_INVALID_ARG for a missing, small or misaligned
 * staging buffer. */
size_t md_batch_staging_bytes(int32_t nsys, const md_system_desc *systems);
int md_batch_prepare_staged(int32_t nsys, const md_system_desc *systems, void *workspace,
                            size_t ws_bytes, void *host_staging, size_t staging_bytes,
                            void *stream);

/* md_step for a batch prepared in `workspace` with the same `systems` (host).  Arrays
 * are the concatenations described above; mode MD_ACCUM_F32, MD_ACCUM_FIXED64 or
 * MD_ACCUM_FIXED_TILE (the last with shapes 0 and 5 only, else MD_ERR_INVALID_ARG).
 * pair_count: device uint64[nsys] or NULL; the unique within-cutoff pairs of every
 * force evaluation are added to it (the caller zeroes it).  Makes no host<->device
 * copies and no allocation, so a sequence of calls can be captured in a CUDA graph
 * (after one call outside the capture). */
int md_batch_step(int32_t nsys, const md_system_desc *systems, double *pos, double *vel,
                  void *forces, int32_t forces_valid, const float *inv_mass, const float *q,
                  const int32_t *type, int32_t mode, double dt_fs, int32_t n_steps,
                  unsigned long long *pair_count, void *workspace, size_t ws_bytes,
                  uint32_t *status, void *stream);

/*
 * Kernel shapes of the batched force launches.  A shape is a performance choice only:
 * every shape finds the same pairs, and in MD_ACCUM_FIXED64 gives the same bits.
 *   0  default: the cluster-pair kernel (MD_ALGO_CLUSTER)
 *   1  half-shell kernel, 4 warps per block, 256 (F32) or 128 (FIXED64) buffered pairs
 *      per warp
 *   2  half-shell kernel, 2 warps per block, 256 buffered pairs per warp
 *   3  half-shell kernel, 8 warps per block, 256 buffered pairs per warp
 *   4  half-shell kernel, 4 warps per block, 128 buffered pairs per warp
 *   5  the cluster-pair kernel on a persistent grid: about one wave of blocks, each
 *      taking cell pairs from a counter until none are left
 * The half-shell buffer holds the filter's survivors of one 32x32 block of candidate
 * pairs (the paper's queue between distance and force stages, Section IV); a block that
 * keeps more is processed in several passes.  More warps per block share the block's
 * staged cells among more candidate blocks; fewer give more blocks per SM for small
 * cells.
 */
#define MD_BATCH_SHAPES 6
typedef struct md_batch_tuning {
    int32_t shape_regular; /* launch over the systems with >= 3 cells on every axis */
    int32_t shape_small;   /* launch over the systems with an axis of 2 cells */
} md_batch_tuning;

/* md_batch_step with the force launches' shapes chosen by `tuning` (host; NULL = both
 * 0).  MD_ERR_INVALID_ARG for a shape outside 0 .. MD_BATCH_SHAPES-1. */
int md_batch_step_tuned(int32_t nsys, const md_system_desc *systems, double *pos, double *vel,
                        void *forces, int32_t forces_valid, const float *inv_mass,
                        const float *q, const int32_t *type, int32_t mode, double dt_fs,
                        int32_t n_steps, unsigned long long *pair_count, void *workspace,
                        size_t ws_bytes, uint32_t *status, const md_batch_tuning *tuning,
                        void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MD_NONBONDED_H */
