/*
 * oracle.c -- plain, single-threaded FP64 reference of the cutoff non-bonded
 * force path.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg call it; the product path never does.  It shares
 * no code, header, table or constant with the CUDA library.
 *
 * What it computes (paper: Section II.A):
 *   Eq. 1  F_LJ = (A/|r|^14 - B/|r|^8) * r
 *   Eq. 2  F_CL = k*q1*q2/|r|^3 * r
 *   cutoff: Eq. 1-2 are evaluated only for pairs closer than the cutoff radius;
 *           beyond it the LJ force is 0 and long-range Coulomb is left out
 *           (the paper leaves it to the host CPU).  The test is strict: r^2 < rc^2.
 *   cell list: cells of edge >= rc, so the partners of an atom lie in its
 *           3x3x3 neighbour cells (Fig. 2 caption, Algorithm 1).
 * Readings where the paper is silent:
 *   - r = x_i - x_j under the minimum-image convention of a periodic box, and
 *     F above is the force on atom i (atom j gets -F).
 *   - Energies are the potentials whose minus gradients are Eq. 1-2:
 *     U_LJ = A/(12 r^12) - B/(6 r^6),  U_C = k q1 q2 / r;  virial W = sum f*r^2
 *     where F = f*r.
 *   - Cells per axis n_d = max(1, floor(L_d/rc)); a coordinate is wrapped as
 *     w = x - L*floor(x/L) (then folded into [0,L)), its cell index is
 *     floor(w * (n_d/L_d)) clamped to [0, n_d-1].  Atoms of a cell are kept in
 *     ascending input order.  When n_d <= 2 the 3x3x3 stencil names the same
 *     cell more than once; each distinct cell is visited once.
 *   - Velocity Verlet (kick-drift-kick) advances the motion (the paper only
 *     says the motion is updated after the forces, Section I / II.A).
 *
 * Two independent force routines: orc_forces_cells (Algorithm 1 loop order,
 * full shell: each pair is met from both sides) and orc_forces_brute (all
 * pairs i<j).  Units: A, fs, amu, e, kcal/mol.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* (kcal/mol/A)/amu in A/fs^2 */
#define ORC_ACCEL 4.184e-4

/* ------------------------------------------------------------------ cells */

int orc_cell_dims(const double *L, double rc, int *dims)
{
    for (int d = 0; d < 3; ++d) {
        if (!(L[d] > 0.0) || !(rc > 0.0)) return -1;
        double nd = floor(L[d] / rc);
        dims[d] = nd < 1.0 ? 1 : (int)nd;
    }
    return 0;
}

static double wrap_coord(double x, double L)
{
    double w = x - L * floor(x / L);
    if (w < 0.0) w += L;
    if (w >= L) w -= L;
    return w;
}

static int cell_coord(double w, int nc, double L)
{
    double inv_edge = (double)nc / L;
    double f = floor(w * inv_edge);
    int c = f < 0.0 ? 0 : (f > (double)(nc - 1) ? nc - 1 : (int)f);
    return c;
}

/* Cell index of every atom, cell_start[ncell+1] and order[n] (atoms of cell c
 * are order[cell_start[c] .. cell_start[c+1]-1], ascending input index). */
int orc_build_cells(int n, const double *pos, const double *L, const int *dims,
                    int *cell_of, int *cell_start, int *order)
{
    int ncell = dims[0] * dims[1] * dims[2];
    for (int i = 0; i < n; ++i) {
        int c[3];
        for (int d = 0; d < 3; ++d)
            c[d] = cell_coord(wrap_coord(pos[3 * i + d], L[d]), dims[d], L[d]);
        cell_of[i] = c[0] + dims[0] * (c[1] + dims[1] * c[2]);
    }
    for (int c = 0; c <= ncell; ++c) cell_start[c] = 0;
    for (int i = 0; i < n; ++i) cell_start[cell_of[i] + 1]++;
    for (int c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
    int *cursor = (int *)malloc(sizeof(int) * (size_t)(ncell > 0 ? ncell : 1));
    if (!cursor) return -2;
    for (int c = 0; c < ncell; ++c) cursor[c] = cell_start[c];
    for (int i = 0; i < n; ++i) order[cursor[cell_of[i]]++] = i;
    free(cursor);
    return 0;
}

/* Distinct neighbour cells of cell (cx,cy,cz) over the 3x3x3 stencil. */
static int neighbour_cells(const int *dims, int cx, int cy, int cz, int *out)
{
    int m = 0;
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                int x = ((cx + ox) % dims[0] + dims[0]) % dims[0];
                int y = ((cy + oy) % dims[1] + dims[1]) % dims[1];
                int z = ((cz + oz) % dims[2] + dims[2]) % dims[2];
                int c = x + dims[0] * (y + dims[1] * z);
                int seen = 0;
                for (int k = 0; k < m; ++k) seen |= (out[k] == c);
                if (!seen) out[m++] = c;
            }
    return m;
}

/* ------------------------------------------------------------- pair terms */

static void min_image(const double *xi, const double *xj, const double *L, double *d)
{
    for (int k = 0; k < 3; ++k) {
        double t = xi[k] - xj[k];
        d[k] = t - L[k] * floor(t / L[k] + 0.5);
    }
}

typedef struct {
    double f;    /* F = f * r (Eq. 1 + Eq. 2 scalar factor) */
    double f_lj; /* Eq. 1 factor alone */
    double f_cl; /* Eq. 2 factor alone */
    double u_lj, u_cl;
    double cond; /* |A| r^-13 + |B| r^-7 + |k q1 q2| r^-2: size of the terms */
} pair_terms;

static pair_terms pair_eval(double r2, double A, double B, double kqq)
{
    pair_terms t;
    double r = sqrt(r2);
    double ir2 = 1.0 / r2;
    double ir6 = ir2 * ir2 * ir2;
    double ir8 = ir6 * ir2;
    double ir14 = ir8 * ir6;
    t.f_lj = A * ir14 - B * ir8;    /* Eq. 1: A/|r|^14 - B/|r|^8 */
    t.f_cl = kqq * ir2 / r;         /* Eq. 2: k q1 q2 / |r|^3     */
    t.f = t.f_lj + t.f_cl;
    t.u_lj = A / 12.0 * ir6 * ir6 - B / 6.0 * ir6;
    t.u_cl = kqq / r;
    t.cond = (fabs(A) * ir14 + fabs(B) * ir8 + fabs(kqq) * ir2 / r) * r;
    return t;
}

/* Force on atom i from atom j (positions as given, minimum image), for tests. */
int orc_pair(const double *xi, const double *xj, const double *L, double qi, double qj,
             double A, double B, double k, double rc, double *F_out, double *u_out)
{
    double d[3];
    min_image(xi, xj, L, d);
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    F_out[0] = F_out[1] = F_out[2] = 0.0;
    if (u_out) u_out[0] = u_out[1] = 0.0;
    if (!(r2 < rc * rc)) return 0;
    pair_terms t = pair_eval(r2, A, B, k * qi * qj);
    for (int c = 0; c < 3; ++c) F_out[c] = t.f * d[c];
    if (u_out) { u_out[0] = t.u_lj; u_out[1] = t.u_cl; }
    return 1;
}

/* --------------------------------------------------- O1: cell list (Alg. 1) */

typedef struct {
    int n;
    double *w;     /* wrapped positions [n*3] */
    int dims[3];
    int ncell;
    int *cell_of, *cell_start, *order;
} cell_list;

static void cl_free(cell_list *cl)
{
    free(cl->w); free(cl->cell_of); free(cl->cell_start); free(cl->order);
}

static int cl_make(cell_list *cl, int n, const double *pos, const double *L, double rc)
{
    memset(cl, 0, sizeof(*cl));
    cl->n = n;
    if (orc_cell_dims(L, rc, cl->dims)) return -1;
    cl->ncell = cl->dims[0] * cl->dims[1] * cl->dims[2];
    cl->w = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    cl->cell_of = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    cl->order = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    cl->cell_start = (int *)malloc(sizeof(int) * (size_t)(cl->ncell + 1));
    if (!cl->w || !cl->cell_of || !cl->order || !cl->cell_start) { cl_free(cl); return -2; }
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) cl->w[3 * i + d] = wrap_coord(pos[3 * i + d], L[d]);
    return orc_build_cells(n, cl->w, L, cl->dims, cl->cell_of, cl->cell_start, cl->order);
}

/*
 * Full-shell cell-list forces in Algorithm 1's loop order:
 *   foreach cell / foreach neighbour cell / foreach atom i of the home cell:
 *     total = 0; foreach atom j of the neighbour cell: if r^2 < rc^2: total += F_ij
 *     F_i += total
 * Every pair is met twice (once from each side), so energies and the virial
 * take half of each meeting.  Outputs (any may be NULL except F):
 *   F[n*3], energy[3] = {E_LJ, E_C, W}, cond[n] = sum over partners of the
 *   term sizes, fabs_sum[n] = sum over partners of |F_ij|, npairs = unique pairs,
 *   energy_abs[3] = the same sums as energy[] taken over absolute term sizes.
 */
int orc_forces_cells(int n, const double *pos, const double *q, const int *type,
                     const double *L, int ntypes, const double *A, const double *B,
                     double k, double rc, double *F, double *energy, double *cond,
                     double *fabs_sum, long long *npairs, double *energy_abs)
{
    cell_list cl;
    int rcode = cl_make(&cl, n, pos, L, rc);
    if (rcode) return rcode;
    double rc2 = rc * rc;
    double e_lj = 0.0, e_cl = 0.0, vir = 0.0;
    double a_lj = 0.0, a_cl = 0.0, a_vir = 0.0;
    long long ordered = 0;
    for (int i = 0; i < 3 * n; ++i) F[i] = 0.0;
    if (cond) for (int i = 0; i < n; ++i) cond[i] = 0.0;
    if (fabs_sum) for (int i = 0; i < n; ++i) fabs_sum[i] = 0.0;
    int nb[27];
    for (int cz = 0; cz < cl.dims[2]; ++cz)
    for (int cy = 0; cy < cl.dims[1]; ++cy)
    for (int cx = 0; cx < cl.dims[0]; ++cx) {
        int home = cx + cl.dims[0] * (cy + cl.dims[1] * cz);
        int m = neighbour_cells(cl.dims, cx, cy, cz, nb);
        for (int kc = 0; kc < m; ++kc) {
            int nbr = nb[kc];
            for (int a = cl.cell_start[home]; a < cl.cell_start[home + 1]; ++a) {
                int i = cl.order[a];
                double total[3] = {0.0, 0.0, 0.0};
                for (int b = cl.cell_start[nbr]; b < cl.cell_start[nbr + 1]; ++b) {
                    int j = cl.order[b];
                    if (j == i) continue;
                    double d[3];
                    min_image(&cl.w[3 * i], &cl.w[3 * j], L, d);
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (!(r2 < rc2)) continue;
                    int tp = type[i] * ntypes + type[j];
                    pair_terms t = pair_eval(r2, A[tp], B[tp], k * q[i] * q[j]);
                    for (int c = 0; c < 3; ++c) total[c] += t.f * d[c];
                    e_lj += 0.5 * t.u_lj;
                    e_cl += 0.5 * t.u_cl;
                    vir += 0.5 * t.f * r2;
                    a_lj += 0.5 * (fabs(A[tp]) / 12.0 * pow(r2, -6.0) + fabs(B[tp]) / 6.0 * pow(r2, -3.0));
                    a_cl += 0.5 * fabs(t.u_cl);
                    a_vir += 0.5 * t.cond * sqrt(r2);
                    if (cond) cond[i] += t.cond;
                    if (fabs_sum) fabs_sum[i] += fabs(t.f) * sqrt(r2);
                    ordered++;
                }
                for (int c = 0; c < 3; ++c) F[3 * i + c] += total[c];
            }
        }
    }
    if (energy) { energy[0] = e_lj; energy[1] = e_cl; energy[2] = vir; }
    if (energy_abs) { energy_abs[0] = a_lj; energy_abs[1] = a_cl; energy_abs[2] = a_vir; }
    if (npairs) *npairs = ordered / 2;
    cl_free(&cl);
    return 0;
}

/* Forces on a chosen subset of atoms only (cell list, full shell).  For
 * spot checks of large systems: cost is ~27 cells of partners per atom. */
int orc_forces_atoms(int n, const double *pos, const double *q, const int *type,
                     const double *L, int ntypes, const double *A, const double *B,
                     double k, double rc, int nsel, const int *sel, double *F_sel,
                     double *cond_sel, int *npart_sel)
{
    cell_list cl;
    int rcode = cl_make(&cl, n, pos, L, rc);
    if (rcode) return rcode;
    double rc2 = rc * rc;
    int nb[27];
    for (int s = 0; s < nsel; ++s) {
        int i = sel[s];
        int c = cl.cell_of[i];
        int cx = c % cl.dims[0], cy = (c / cl.dims[0]) % cl.dims[1], cz = c / (cl.dims[0] * cl.dims[1]);
        int m = neighbour_cells(cl.dims, cx, cy, cz, nb);
        double tot[3] = {0.0, 0.0, 0.0}, cd = 0.0;
        int np = 0;
        for (int kc = 0; kc < m; ++kc) {
            int nbr = nb[kc];
            for (int b = cl.cell_start[nbr]; b < cl.cell_start[nbr + 1]; ++b) {
                int j = cl.order[b];
                if (j == i) continue;
                double d[3];
                min_image(&cl.w[3 * i], &cl.w[3 * j], L, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (!(r2 < rc2)) continue;
                int tp = type[i] * ntypes + type[j];
                pair_terms t = pair_eval(r2, A[tp], B[tp], k * q[i] * q[j]);
                for (int cc = 0; cc < 3; ++cc) tot[cc] += t.f * d[cc];
                cd += t.cond;
                np++;
            }
        }
        for (int cc = 0; cc < 3; ++cc) F_sel[3 * s + cc] = tot[cc];
        if (cond_sel) cond_sel[s] = cd;
        if (npart_sel) npart_sel[s] = np;
    }
    cl_free(&cl);
    return 0;
}

/* ------------------------------------------------------ O2: brute force */

int orc_forces_brute(int n, const double *pos, const double *q, const int *type,
                     const double *L, int ntypes, const double *A, const double *B,
                     double k, double rc, double *F, double *energy, long long *npairs)
{
    double rc2 = rc * rc;
    double e_lj = 0.0, e_cl = 0.0, vir = 0.0;
    long long np = 0;
    for (int i = 0; i < 3 * n; ++i) F[i] = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double d[3];
            min_image(&pos[3 * i], &pos[3 * j], L, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < rc2)) continue;
            int tp = type[i] * ntypes + type[j];
            pair_terms t = pair_eval(r2, A[tp], B[tp], k * q[i] * q[j]);
            for (int c = 0; c < 3; ++c) {
                F[3 * i + c] += t.f * d[c];
                F[3 * j + c] -= t.f * d[c];
            }
            e_lj += t.u_lj;
            e_cl += t.u_cl;
            vir += t.f * r2;
            np++;
        }
    if (energy) { energy[0] = e_lj; energy[1] = e_cl; energy[2] = vir; }
    if (npairs) *npairs = np;
    return 0;
}

/* Pairs whose squared distance lies within `window` of rc^2: where an FP32
 * filter may legitimately decide differently from this FP64 one.  Writes up to
 * max_out (i, j) with i<j and their r^2; returns how many exist in total. */
long long orc_boundary_pairs(int n, const double *pos, const double *L, double rc,
                             double window, int max_out, int *ij, double *r2_out)
{
    cell_list cl;
    if (cl_make(&cl, n, pos, L, rc)) return -1;
    double rc2 = rc * rc;
    long long cnt = 0;
    int nb[27];
    for (int c = 0; c < cl.ncell; ++c) {
        int cx = c % cl.dims[0], cy = (c / cl.dims[0]) % cl.dims[1], cz = c / (cl.dims[0] * cl.dims[1]);
        int m = neighbour_cells(cl.dims, cx, cy, cz, nb);
        for (int kc = 0; kc < m; ++kc)
            for (int a = cl.cell_start[c]; a < cl.cell_start[c + 1]; ++a)
                for (int b = cl.cell_start[nb[kc]]; b < cl.cell_start[nb[kc] + 1]; ++b) {
                    int i = cl.order[a], j = cl.order[b];
                    if (!(i < j)) continue;
                    double d[3];
                    min_image(&cl.w[3 * i], &cl.w[3 * j], L, d);
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (fabs(r2 - rc2) <= window) {
                        if (cnt < max_out) {
                            ij[2 * cnt] = i; ij[2 * cnt + 1] = j; r2_out[cnt] = r2;
                        }
                        cnt++;
                    }
                }
    }
    cl_free(&cl);
    return cnt;
}

/* ------------------------------------------------------- velocity Verlet */

double orc_kinetic_energy(int n, const double *vel, const double *inv_mass)
{
    double ke = 0.0;
    for (int i = 0; i < n; ++i) {
        double v2 = vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] + vel[3 * i + 2] * vel[3 * i + 2];
        ke += 0.5 * v2 / inv_mass[i] / ORC_ACCEL;
    }
    return ke;
}

/*
 * n_steps of kick-drift-kick velocity Verlet:
 *   v += dt/2 * a(x);  x += dt * v;  x <- wrap(x);  F = F(x);  v += dt/2 * a(x)
 * with a = F * inv_mass * 4.184e-4.  Each update is one correctly rounded fused
 * multiply-add (C99 fma): v = fma(F, c, v) with c = dt/2 * inv_mass * 4.184e-4
 * (evaluated left to right) and x = fma(dt, v, x).  F holds F(x) on entry when f_valid is
 * non-zero (else it is computed first) and F(x_final) on exit.  When
 * f32_positions is non-zero the forces are evaluated at the positions rounded
 * to float32 (the state itself stays float64).  energy_log (may be NULL) gets
 * {E_LJ, E_C, KE, W} after every step.
 */
int orc_vv_steps(int n, double *pos, double *vel, double *F, int f_valid,
                 const double *inv_mass, const double *q, const int *type,
                 const double *L, int ntypes, const double *A, const double *B,
                 double k, double rc, double dt, int n_steps, int f32_positions,
                 double *energy_log)
{
    double *xf = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!xf) return -2;
    double en[3];
    int rcode = 0;
#define ORC_FORCES()                                                              \
    do {                                                                          \
        for (int i_ = 0; i_ < 3 * n; ++i_)                                        \
            xf[i_] = f32_positions ? (double)(float)pos[i_] : pos[i_];            \
        rcode = orc_forces_cells(n, xf, q, type, L, ntypes, A, B, k, rc, F, en,   \
                                 NULL, NULL, NULL, NULL);                         \
    } while (0)
    if (!f_valid) ORC_FORCES();
    for (int s = 0; s < n_steps && rcode == 0; ++s) {
        for (int i = 0; i < n; ++i) {
            const double kf = 0.5 * dt * inv_mass[i] * ORC_ACCEL;
            for (int c = 0; c < 3; ++c) {
                vel[3 * i + c] = fma(F[3 * i + c], kf, vel[3 * i + c]);
                pos[3 * i + c] = wrap_coord(fma(dt, vel[3 * i + c], pos[3 * i + c]), L[c]);
            }
        }
        ORC_FORCES();
        for (int i = 0; i < n; ++i) {
            const double kf = 0.5 * dt * inv_mass[i] * ORC_ACCEL;
            for (int c = 0; c < 3; ++c)
                vel[3 * i + c] = fma(F[3 * i + c], kf, vel[3 * i + c]);
        }
        if (energy_log) {
            energy_log[4 * s + 0] = en[0];
            energy_log[4 * s + 1] = en[1];
            energy_log[4 * s + 2] = orc_kinetic_energy(n, vel, inv_mass);
            energy_log[4 * s + 3] = en[2];
        }
    }
#undef ORC_FORCES
    free(xf);
    return rcode;
}
