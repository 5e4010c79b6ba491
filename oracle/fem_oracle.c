/*
 * fem_oracle.c -- plain, slow, FP64 reference of the explicit element-by-
 * element enthalpy step for transient heat conduction with phase change on
 * linear tetrahedra (Tavakoli, "Improvement cache efficiency of explicit
 * finite element procedure and its application to parallel casting
 * solidification simulation", Sections 2-4.1.2).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it; the product library never does.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * Deliberately naive: every element keeps its dense 4x4 conductance matrix
 * K^e (the paper stores exactly this, Eq. 18 and the text after it), global
 * node arrays, one thread, FP64 throughout, no blocking, no reordering.
 *
 * What it computes (each function cites the passage it follows):
 *   - K^e = k V [grad N_i . grad N_j] of the linear tet (Galerkin, Eq. 9),
 *   - row-sum lumped capacities (Section 3, text after Eq. 9),
 *   - the enthalpy E(T) = C T + Lc f_l(T) with a linear liquid fraction
 *     between solidus and liquidus (Eqs. 5 and 11) and its exact inverse,
 *   - Robin faces -k dT/dn = q + h (T - T_inf) (Eq. 4) with the consistent
 *     Galerkin face matrix h A / 12 (1 + delta_ij) and load A/3 (h T_inf - q),
 *   - the explicit update E += dt (F - K T) (Eq. 14 with theta = 0 in Eq. 10,
 *     written for the enthalpy unknown of Eq. 5),
 *   - alternatively the paper's apparent-heat-capacity form (Eqs. 6-7,
 *     Lemmon's method) with T as the unknown: C_app (T^{n+1} - T^n) / dt =
 *     F - K T^n, C_app lumped from each element's apparent specific heat,
 *   - Dirichlet nodes (Eq. 3) held at E(T_D),
 *   - optional temperature-dependent conductivity k(T) per material (Eq. 9
 *     allows K(T)): a piecewise-linear table evaluated at the element's mean
 *     temperature at step n, K^e(T) = k(T_mean) x (K^e for k = 1),
 *   - the cast-mold interface of Eq. 8: faces of two regions meshed
 *     separately, each exchanging h_i (T_sister - T) with the mean
 *     temperature of its sister, the nearest face of the other region
 *     (found once, Section 3),
 *   - FP64 energy bookkeeping: U = sum E, cumulative boundary heat, latent
 *     heat still to be released,
 *   - a Gershgorin stable time step for the explicit scheme (reading of
 *     Eq. 13, which gives the bound only up to an unstated constant).
 *
 * Parity pins (tests/test_oracle_*.py): closed-form unit tet, an independent
 * barycentric-solve stiffness, the linear patch test, lumped sums, T(E) round
 * trips, adiabatic energy conservation, the first-step Robin energy change,
 * uniform equilibrium, the erfc and erf slab solutions, the Neumann two-phase
 * Stefan solution and the eigenvalue stability limit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_KT_MAX 16
#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

typedef struct oracle_problem {
    int64_t n_nodes, n_tets, n_faces;
    double *xyz;     /* [N][3] coordinates (interface centroids and areas) */
    /* element data */
    int32_t *tets;   /* [E][4], re-oriented to positive volume */
    double *Ke;      /* [E][4][4] dense conductance matrices */
    double *Kg;      /* [E][4][4] the same for k = 1 (geometric part) */
    int32_t *emat;   /* [E] material id */
    /* optional conductivity tables k(T) per material (Eq. 9's K(T)):
     * kt_n[m] points (kt_T ascending, kt_k), 0 = constant k */
    int32_t n_mat;
    double *mats;    /* [n_mat][6] rho, c, k, latent, T_solidus, T_liquidus */
    /* formulation: 0 = enthalpy (Eq. 5), 1 = apparent heat capacity by
     * Lemmon's method (Eqs. 6-7) with T as the unknown */
    int form;
    double *Tst;     /* [N] temperatures, the unknowns of formulation 1 */
    double *cap;     /* [N] lumped apparent capacity of the current step */
    int32_t *kt_n;
    double *kt_T, *kt_k;  /* [n_mat][ORACLE_KT_MAX] */
    double *vol;     /* [E] */
    /* lumped nodal data */
    double *C;       /* sensible heat capacity, J/K */
    double *m;       /* lumped mass, kg */
    double *Lc;      /* latent capacity, J */
    double *Ts, *Tl; /* phase-change range of the node (unused if Lc == 0) */
    /* Robin faces */
    int32_t *faces;  /* [F][3] */
    double *fh, *ftinf, *fq, *farea;
    /* cast-mold interface (Eq. 8): faces of side 0 then side 1; each face
     * sees the mean temperature of its sister, the other side's face with
     * the nearest centroid, as its ambient temperature */
    int64_t n_if;
    int32_t *if_faces;   /* [n_if][3] */
    double *if_h, *if_area;
    int64_t *if_sister;  /* index into the interface list */
    /* Dirichlet */
    uint8_t *is_dir;
    double *T_dir;
    /* state */
    double *E, *T, *R;
    int64_t step;
    double time;
    double U0;       /* total enthalpy at the initial condition */
    double Qb;       /* cumulative heat that entered through the Robin faces */
} oracle_problem;

/* ------------------------------------------------------------------------ */
/* Enthalpy relation (Eqs. 5 and 11, linear liquid fraction)                 */
/* ------------------------------------------------------------------------ */

/* Liquid fraction f_l(T): 0 below solidus, 1 above liquidus, linear between.
 * In the isothermal limit (Ts == Tl) a node exactly at the melting point is
 * taken as liquid. */
double oracle_liquid_fraction(double T, double Ts, double Tl)
{
    if (Tl <= Ts) return T >= Ts ? 1.0 : 0.0;
    if (T <= Ts) return 0.0;
    if (T >= Tl) return 1.0;
    return (T - Ts) / (Tl - Ts);
}

/* Nodal enthalpy content E(T) = C T + Lc f_l(T), datum E = 0 at T = 0 K. */
double oracle_E_from_T(double T, double C, double Lc, double Ts, double Tl)
{
    if (Lc <= 0.0) return C * T;
    return C * T + Lc * oracle_liquid_fraction(T, Ts, Tl);
}

/* Inverse of the monotone piecewise-linear E(T). */
double oracle_T_from_E(double E, double C, double Lc, double Ts, double Tl)
{
    if (Lc <= 0.0) return E / C;
    double E_solid = C * Ts;           /* enthalpy of solid at the solidus */
    double E_liquid = C * Tl + Lc;     /* enthalpy of liquid at the liquidus */
    if (E <= E_solid) return E / C;
    if (E >= E_liquid) return (E - Lc) / C;
    if (Tl <= Ts) return Ts;           /* isothermal: latent plateau */
    /* mushy zone: dE/dT = C + Lc / (Tl - Ts) */
    return Ts + (E - E_solid) / (C + Lc / (Tl - Ts));
}

/* ------------------------------------------------------------------------ */
/* Element matrix (Eq. 9, standard Galerkin on the linear tet)              */
/* ------------------------------------------------------------------------ */

static double det3(const double J[3][3])
{
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
         - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
         + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

/* x: the 4 corners, x[3*a + d].  Writes K[4*a + b] = k V gradN_a . gradN_b
 * and the signed volume V = det(J)/6 with J's columns x_b-x_a, x_c-x_a,
 * x_d-x_a.  The barycentric coordinates of corners b, c, d are
 * J^{-1} (x - x_a), so their gradients are the rows of J^{-1}; the gradient
 * of corner a is minus their sum.  The matrix uses |V|. */
int oracle_tet_matrix(const double *x, double k, double *K, double *vol)
{
    double J[3][3];
    for (int d = 0; d < 3; d++)
        for (int c = 0; c < 3; c++)
            J[d][c] = x[3 * (c + 1) + d] - x[d];
    double det = det3(J);
    *vol = det / 6.0;
    if (det == 0.0) return ORACLE_EINVAL;
    /* inverse by cofactors: Jinv[r][c] = cof(J)[c][r] / det */
    double Jinv[3][3];
    Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    double g[4][3];
    for (int d = 0; d < 3; d++) {
        g[1][d] = Jinv[0][d];
        g[2][d] = Jinv[1][d];
        g[3][d] = Jinv[2][d];
        g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
    }
    double kv = k * fabs(*vol);
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++)
            K[4 * a + b] = kv * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
    return ORACLE_OK;
}

static double tri_area(const double *xa, const double *xb, const double *xc)
{
    double u[3], v[3];
    for (int d = 0; d < 3; d++) { u[d] = xb[d] - xa[d]; v[d] = xc[d] - xa[d]; }
    double n0 = u[1] * v[2] - u[2] * v[1];
    double n1 = u[2] * v[0] - u[0] * v[2];
    double n2 = u[0] * v[1] - u[1] * v[0];
    return 0.5 * sqrt(n0 * n0 + n1 * n1 + n2 * n2);
}

/* ------------------------------------------------------------------------ */
/* Problem set-up                                                            */
/* ------------------------------------------------------------------------ */

void oracle_destroy(oracle_problem *p)
{
    if (!p) return;
    free(p->tets); free(p->Ke); free(p->Kg); free(p->emat); free(p->vol);
    free(p->kt_n); free(p->kt_T); free(p->kt_k); free(p->mats); free(p->Tst); free(p->cap);
    free(p->C); free(p->m); free(p->Lc); free(p->Ts); free(p->Tl);
    free(p->faces); free(p->fh); free(p->ftinf); free(p->fq); free(p->farea);
    free(p->if_faces); free(p->if_h); free(p->if_area); free(p->if_sister); free(p->xyz);
    free(p->is_dir); free(p->T_dir);
    free(p->E); free(p->T); free(p->R);
    free(p);
}

/*
 * mats: [n_mat][6] rows (rho, c, k, latent, T_solidus, T_liquidus); latent 0
 * means no phase change.  faces may be NULL if n_faces == 0; q may be NULL
 * (zero flux).  Returns NULL on invalid input (index out of range, degenerate
 * tet, a node carrying two different phase-change ranges) with *status set.
 */
oracle_problem *oracle_create(int64_t n_nodes, const double *xyz,
                              int64_t n_tets, const int32_t *tets, const int32_t *mat,
                              int32_t n_mat, const double *mats,
                              int64_t n_faces, const int32_t *faces,
                              const double *h, const double *t_inf, const double *q,
                              int64_t n_dir, const int32_t *dir_nodes, const double *dir_T,
                              int *status)
{
    *status = ORACLE_EINVAL;
    if (n_nodes <= 0 || n_tets <= 0 || n_faces < 0 || n_dir < 0 || n_mat <= 0) return NULL;
    oracle_problem *p = (oracle_problem *)calloc(1, sizeof(*p));
    if (!p) { *status = ORACLE_ENOMEM; return NULL; }
    p->n_nodes = n_nodes; p->n_tets = n_tets; p->n_faces = n_faces;
    size_t N = (size_t)n_nodes, E = (size_t)n_tets, F = (size_t)n_faces;
    p->xyz = malloc(3 * N * sizeof(double));
    p->tets = malloc(4 * E * sizeof(int32_t));
    p->Ke = malloc(16 * E * sizeof(double));
    p->Kg = malloc(16 * E * sizeof(double));
    p->emat = malloc(E * sizeof(int32_t));
    p->n_mat = n_mat;
    p->mats = malloc((size_t)n_mat * 6 * sizeof(double));
    p->Tst = calloc(N, sizeof(double));
    p->cap = calloc(N, sizeof(double));
    p->kt_n = calloc((size_t)n_mat, sizeof(int32_t));
    p->kt_T = calloc((size_t)n_mat * ORACLE_KT_MAX, sizeof(double));
    p->kt_k = calloc((size_t)n_mat * ORACLE_KT_MAX, sizeof(double));
    p->vol = malloc(E * sizeof(double));
    p->C = calloc(N, sizeof(double));
    p->m = calloc(N, sizeof(double));
    p->Lc = calloc(N, sizeof(double));
    p->Ts = calloc(N, sizeof(double));
    p->Tl = calloc(N, sizeof(double));
    p->faces = malloc((3 * F + 1) * sizeof(int32_t));
    p->fh = malloc((F + 1) * sizeof(double));
    p->ftinf = malloc((F + 1) * sizeof(double));
    p->fq = malloc((F + 1) * sizeof(double));
    p->farea = malloc((F + 1) * sizeof(double));
    p->is_dir = calloc(N, 1);
    p->T_dir = calloc(N, sizeof(double));
    p->E = calloc(N, sizeof(double));
    p->T = calloc(N, sizeof(double));
    p->R = calloc(N, sizeof(double));
    if (!p->xyz || !p->tets || !p->Ke || !p->Kg || !p->emat || !p->kt_n || !p->kt_T || !p->kt_k ||
        !p->mats || !p->Tst || !p->cap ||
        !p->vol || !p->C || !p->m || !p->Lc || !p->Ts || !p->Tl ||
        !p->faces || !p->fh || !p->ftinf || !p->fq || !p->farea || !p->is_dir ||
        !p->T_dir || !p->E || !p->T || !p->R) {
        oracle_destroy(p); *status = ORACLE_ENOMEM; return NULL;
    }
    memcpy(p->xyz, xyz, 3 * N * sizeof(double));
    memcpy(p->mats, mats, (size_t)n_mat * 6 * sizeof(double));
    uint8_t *has_range = calloc(N, 1);
    if (!has_range) { oracle_destroy(p); *status = ORACLE_ENOMEM; return NULL; }

    for (size_t e = 0; e < E; e++) {
        int32_t n[4];
        for (int a = 0; a < 4; a++) {
            n[a] = tets[4 * e + a];
            if (n[a] < 0 || n[a] >= n_nodes) goto bad;
        }
        if (mat[e] < 0 || mat[e] >= n_mat) goto bad;
        const double *M = mats + 6 * (size_t)mat[e];
        double rho = M[0], c = M[1], k = M[2], L = M[3], Ts = M[4], Tl = M[5];
        double x[12];
        for (int a = 0; a < 4; a++)
            for (int d = 0; d < 3; d++) x[3 * a + d] = xyz[3 * (size_t)n[a] + d];
        double V;
        if (oracle_tet_matrix(x, k, p->Ke + 16 * e, &V) != ORACLE_OK) goto bad;
        /* degenerate-tet test against the mean edge length */
        double lsum = 0.0;
        for (int a = 0; a < 4; a++)
            for (int b = a + 1; b < 4; b++) {
                double d0 = x[3 * a] - x[3 * b], d1 = x[3 * a + 1] - x[3 * b + 1],
                       d2 = x[3 * a + 2] - x[3 * b + 2];
                lsum += sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            }
        double l = lsum / 6.0;
        if (fabs(V) < 1e-12 * l * l * l) goto bad;
        if (V < 0.0) { int32_t t = n[2]; n[2] = n[3]; n[3] = t; }
        /* K^e is unchanged by swapping two corners together with its rows and
         * columns; recompute it on the re-oriented tet for clarity. */
        for (int a = 0; a < 4; a++)
            for (int d = 0; d < 3; d++) x[3 * a + d] = xyz[3 * (size_t)n[a] + d];
        oracle_tet_matrix(x, k, p->Ke + 16 * e, &V);
        oracle_tet_matrix(x, 1.0, p->Kg + 16 * e, &V);
        p->emat[e] = mat[e];
        p->vol[e] = V;
        for (int a = 0; a < 4; a++) p->tets[4 * e + a] = n[a];
        /* row-sum lumping of the consistent capacity rho c V/20 (1 + delta):
         * each row sums to rho c V / 4 */
        for (int a = 0; a < 4; a++) {
            p->C[n[a]] += rho * c * V / 4.0;
            p->m[n[a]] += rho * V / 4.0;
            if (L > 0.0) {
                p->Lc[n[a]] += rho * L * V / 4.0;
                if (has_range[n[a]] && (p->Ts[n[a]] != Ts || p->Tl[n[a]] != Tl)) goto bad;
                p->Ts[n[a]] = Ts; p->Tl[n[a]] = Tl; has_range[n[a]] = 1;
            }
        }
    }
    for (size_t f = 0; f < F; f++) {
        for (int a = 0; a < 3; a++) {
            int32_t v = faces[3 * f + a];
            if (v < 0 || v >= n_nodes) goto bad;
            p->faces[3 * f + a] = v;
        }
        p->fh[f] = h[f];
        p->ftinf[f] = t_inf[f];
        p->fq[f] = q ? q[f] : 0.0;
        p->farea[f] = tri_area(xyz + 3 * (size_t)p->faces[3 * f],
                               xyz + 3 * (size_t)p->faces[3 * f + 1],
                               xyz + 3 * (size_t)p->faces[3 * f + 2]);
    }
    for (int64_t i = 0; i < n_dir; i++) {
        int32_t v = dir_nodes[i];
        if (v < 0 || v >= n_nodes) goto bad;
        p->is_dir[v] = 1;
        p->T_dir[v] = dir_T[i];
    }
    free(has_range);
    *status = ORACLE_OK;
    return p;
bad:
    free(has_range);
    oracle_destroy(p);
    *status = ORACLE_EINVAL;
    return NULL;
}

/* Initial condition, Eq. 2: E_i = E(T0_i); Dirichlet nodes take E(T_D). */
void oracle_set_temperature(oracle_problem *p, const double *T0)
{
    double U = 0.0;
    for (int64_t i = 0; i < p->n_nodes; i++) {
        double T = p->is_dir[i] ? p->T_dir[i] : T0[i];
        p->Tst[i] = T;
        p->E[i] = oracle_E_from_T(T, p->C[i], p->Lc[i], p->Ts[i], p->Tl[i]);
        U += p->E[i];
    }
    p->U0 = U;
    p->Qb = 0.0;
    p->step = 0;
    p->time = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Right-hand side F - K T (Eqs. 4, 9, 15-18)                                */
/* ------------------------------------------------------------------------ */

/* Temperature-dependent conductivity (Eq. 9 allows K(T)): material mt's
 * table of n points (T_j ascending, k_j), linear between points, constant
 * beyond the first and last.  Returns ORACLE_EINVAL for a bad table. */
int oracle_set_conductivity(oracle_problem *p, int32_t mt, int32_t n, const double *T,
                            const double *k)
{
    if (mt < 0 || mt >= p->n_mat || n < 0 || n > ORACLE_KT_MAX) return ORACLE_EINVAL;
    for (int32_t j = 0; j < n; j++) {
        if (!(k[j] > 0.0) || !isfinite(T[j]) || !isfinite(k[j])) return ORACLE_EINVAL;
        if (j > 0 && !(T[j] > T[j - 1])) return ORACLE_EINVAL;
    }
    p->kt_n[mt] = n;
    for (int32_t j = 0; j < n; j++) {
        p->kt_T[ORACLE_KT_MAX * mt + j] = T[j];
        p->kt_k[ORACLE_KT_MAX * mt + j] = k[j];
    }
    return ORACLE_OK;
}

double oracle_conductivity(const oracle_problem *p, int32_t mt, double T)
{
    int32_t n = p->kt_n[mt];
    const double *Tj = p->kt_T + ORACLE_KT_MAX * mt, *kj = p->kt_k + ORACLE_KT_MAX * mt;
    if (T <= Tj[0]) return kj[0];
    if (T >= Tj[n - 1]) return kj[n - 1];
    int32_t j = 0;
    while (T > Tj[j + 1]) j++;
    return kj[j] + (kj[j + 1] - kj[j]) * (T - Tj[j]) / (Tj[j + 1] - Tj[j]);
}

/* R = F - K T for the nodal temperatures T, summing element contributions
 * one element at a time (Eq. 18) and then the Robin faces.  Elements with
 * elem_part[e] != part (and faces with face_part[f] != part) are skipped
 * when the part arrays are given: this is the partial sum of one partition
 * of Eqs. 19-21, whose sum over partitions is Eq. 22.  Returns the heat that
 * entered through the included faces per unit time. */
double oracle_residual_part(const oracle_problem *p, const double *T, double *R,
                            const int32_t *elem_part, const int32_t *face_part,
                            int32_t part)
{
    for (int64_t i = 0; i < p->n_nodes; i++) R[i] = 0.0;
    for (int64_t e = 0; e < p->n_tets; e++) {
        if (elem_part && elem_part[e] != part) continue;
        const int32_t *n = p->tets + 4 * e;
        const int32_t mt = p->emat[e];
        if (p->kt_n[mt] > 0) {
            /* K^e(T) = k(mean element temperature at step n) x geometric part */
            double Tm = (T[n[0]] + T[n[1]] + T[n[2]] + T[n[3]]) / 4.0;
            double kk = oracle_conductivity(p, mt, Tm);
            const double *K = p->Kg + 16 * e;
            for (int a = 0; a < 4; a++) {
                double s = 0.0;
                for (int b = 0; b < 4; b++) s += kk * K[4 * a + b] * T[n[b]];
                R[n[a]] -= s;
            }
            continue;
        }
        const double *K = p->Ke + 16 * e;
        for (int a = 0; a < 4; a++) {
            double s = 0.0;
            for (int b = 0; b < 4; b++) s += K[4 * a + b] * T[n[b]];
            R[n[a]] -= s;
        }
    }
    double qin = 0.0;
    for (int64_t f = 0; f < p->n_faces; f++) {
        if (face_part && face_part[f] != part) continue;
        const int32_t *n = p->faces + 3 * f;
        double hA12 = p->fh[f] * p->farea[f] / 12.0;
        double load = p->farea[f] / 3.0 * (p->fh[f] * p->ftinf[f] - p->fq[f]);
        for (int a = 0; a < 3; a++) {
            double s = 0.0;
            for (int b = 0; b < 3; b++) s += hA12 * (a == b ? 2.0 : 1.0) * T[n[b]];
            double r = load - s;
            R[n[a]] += r;
            qin += r;
        }
    }
    /* interface faces (whole residual only): Robin terms with h = h_i and
     * the sister face's mean temperature as the ambient one, q = 0 */
    if (!face_part)
        for (int64_t f = 0; f < p->n_if; f++) {
            const int32_t *n = p->if_faces + 3 * f;
            const int32_t *sn = p->if_faces + 3 * p->if_sister[f];
            double Tamb = (T[sn[0]] + T[sn[1]] + T[sn[2]]) / 3.0;
            double hA12 = p->if_h[f] * p->if_area[f] / 12.0;
            double load = p->if_area[f] / 3.0 * p->if_h[f] * Tamb;
            for (int a = 0; a < 3; a++) {
                double s = 0.0;
                for (int b = 0; b < 3; b++) s += hA12 * (a == b ? 2.0 : 1.0) * T[n[b]];
                double r = load - s;
                R[n[a]] += r;
                qin += r;
            }
        }
    return qin;
}

/* Interface of Eq. 8 between two regions meshed separately: side-0 faces
 * [n0][3] with coefficients h0, side-1 faces [n1][3] with h1 (each face a
 * face of exactly one tet is not checked here).  The sister of a face is the
 * face of the other side whose centroid is nearest (ties: the lower index),
 * found once, as the paper does at the start of a simulation (Section 3).
 * Returns ORACLE_OK, ORACLE_EINVAL or ORACLE_ENOMEM. */
int oracle_set_interface(oracle_problem *p, int64_t n0, const int32_t *f0, const double *h0,
                         int64_t n1, const int32_t *f1, const double *h1)
{
    if (n0 < 0 || n1 < 0 || (n0 > 0) != (n1 > 0)) return ORACLE_EINVAL;
    free(p->if_faces); free(p->if_h); free(p->if_area); free(p->if_sister);
    p->if_faces = NULL; p->if_h = p->if_area = NULL; p->if_sister = NULL;
    p->n_if = 0;
    if (n0 == 0) return ORACLE_OK;
    int64_t n = n0 + n1;
    p->if_faces = malloc((size_t)n * 3 * sizeof(int32_t));
    p->if_h = malloc((size_t)n * sizeof(double));
    p->if_area = malloc((size_t)n * sizeof(double));
    p->if_sister = malloc((size_t)n * sizeof(int64_t));
    double *cen = malloc((size_t)n * 3 * sizeof(double));
    if (!p->if_faces || !p->if_h || !p->if_area || !p->if_sister || !cen) { free(cen); return ORACLE_ENOMEM; }
    for (int64_t f = 0; f < n; f++) {
        const int32_t *src = f < n0 ? f0 + 3 * f : f1 + 3 * (f - n0);
        for (int a = 0; a < 3; a++) {
            if (src[a] < 0 || src[a] >= p->n_nodes) { free(cen); p->n_if = 0; return ORACLE_EINVAL; }
            p->if_faces[3 * f + a] = src[a];
        }
        p->if_h[f] = f < n0 ? h0[f] : h1[f - n0];
        const double *x0 = p->xyz + 3 * (size_t)src[0], *x1 = p->xyz + 3 * (size_t)src[1],
                     *x2 = p->xyz + 3 * (size_t)src[2];
        p->if_area[f] = tri_area(x0, x1, x2);
        for (int d = 0; d < 3; d++) cen[3 * f + d] = (x0[d] + x1[d] + x2[d]) / 3.0;
    }
    for (int64_t f = 0; f < n; f++) {
        int64_t lo = f < n0 ? n0 : 0, hi = f < n0 ? n : n0;
        int64_t best = -1;
        double bd = 0.0;
        for (int64_t g = lo; g < hi; g++) {
            double dx = cen[3 * g] - cen[3 * f], dy = cen[3 * g + 1] - cen[3 * f + 1],
                   dz = cen[3 * g + 2] - cen[3 * f + 2];
            double d = dx * dx + dy * dy + dz * dz;
            if (best < 0 || d < bd) { best = g; bd = d; }
        }
        p->if_sister[f] = best;
    }
    free(cen);
    p->n_if = n;
    return ORACLE_OK;
}

int64_t oracle_interface_sister(const oracle_problem *p, int64_t f)
{
    return (f >= 0 && f < p->n_if) ? p->if_sister[f] : -1;
}

double oracle_residual(const oracle_problem *p, const double *T, double *R)
{
    return oracle_residual_part(p, T, R, NULL, NULL, 0);
}

/* ------------------------------------------------------------------------ */
/* Explicit step (Eq. 14 with theta = 0, enthalpy form of Eq. 5)             */
/* ------------------------------------------------------------------------ */

void oracle_temperatures(const oracle_problem *p, double *T)
{
    if (p->form == 1) {
        memcpy(T, p->Tst, (size_t)p->n_nodes * sizeof(double));
        return;
    }
    for (int64_t i = 0; i < p->n_nodes; i++)
        T[i] = oracle_T_from_E(p->E[i], p->C[i], p->Lc[i], p->Ts[i], p->Tl[i]);
}

/* Apparent specific heat of element e by Lemmon's method (Eq. 7): the
 * ratio of the gradient magnitudes of the specific enthalpy H(T) = c T +
 * L f_l(T) of the element's material and of T, both interpolated linearly
 * from the nodal values.  With K_g the k = 1 element matrix (zero row sums,
 * off-diagonals -w_ab), |grad x|^2 V = x^T K_g x = sum_{a<b} w_ab (x_a -
 * x_b)^2, so cp = sqrt(sum w (H_a - H_b)^2 / sum w (T_a - T_b)^2).  When T
 * is uniform over the element (every difference below a micro-kelvin),
 * dH/dT at the mean temperature is taken instead. */
double oracle_apparent_cp(const oracle_problem *p, int64_t e, const double *T)
{
    const double *M = p->mats + 6 * (size_t)p->emat[e];
    double c = M[1], L = M[3], Ts = M[4], Tl = M[5];
    if (!(L > 0.0)) return c;
    const int32_t *n = p->tets + 4 * e;
    const double *K = p->Kg + 16 * e;
    double H[4];
    for (int a = 0; a < 4; a++) H[a] = c * T[n[a]] + L * oracle_liquid_fraction(T[n[a]], Ts, Tl);
    double num = 0.0, den = 0.0, wsum = 0.0;
    for (int a = 0; a < 4; a++)
        for (int b = a + 1; b < 4; b++) {
            double w = -K[4 * a + b], dH = H[a] - H[b], dT = T[n[a]] - T[n[b]];
            num += w * dH * dH;
            den += w * dT * dT;
            wsum += w;
        }
    if (den > 1e-12 * wsum) return sqrt(num / den);
    double Tm = (T[n[0]] + T[n[1]] + T[n[2]] + T[n[3]]) / 4.0;
    return (Tm >= Ts && Tm < Tl) ? c + L / (Tl - Ts) : c;
}

/* Formulation 1 (apparent capacity) is defined for phase-change ranges of
 * positive width only. */
int oracle_set_formulation(oracle_problem *p, int form)
{
    if (form != 0 && form != 1) return ORACLE_EINVAL;
    if (form == 1)
        for (int32_t m = 0; m < p->n_mat; m++)
            if (p->mats[6 * m + 3] > 0.0 && !(p->mats[6 * m + 5] > p->mats[6 * m + 4])) return ORACLE_EINVAL;
    p->form = form;
    for (int64_t i = 0; i < p->n_nodes; i++)
        p->Tst[i] = oracle_T_from_E(p->E[i], p->C[i], p->Lc[i], p->Ts[i], p->Tl[i]);
    return ORACLE_OK;
}

/* One explicit step of formulation 1 (Eqs. 9, 10 with theta = 0 and the
 * lumped apparent capacity C_i = sum_e rho V / 4 cp_app,e of step n). */
static void oracle_step_apparent(oracle_problem *p, double dt)
{
    double qin = oracle_residual(p, p->Tst, p->R);
    p->Qb += dt * qin;
    for (int64_t i = 0; i < p->n_nodes; i++) p->cap[i] = 0.0;
    for (int64_t e = 0; e < p->n_tets; e++) {
        double rho = p->mats[6 * (size_t)p->emat[e]];
        double cp = oracle_apparent_cp(p, e, p->Tst);
        for (int a = 0; a < 4; a++) p->cap[p->tets[4 * e + a]] += rho * p->vol[e] / 4.0 * cp;
    }
    for (int64_t i = 0; i < p->n_nodes; i++) {
        if (p->is_dir[i]) p->Tst[i] = p->T_dir[i];
        else p->Tst[i] += dt * p->R[i] / p->cap[i];
        p->E[i] = oracle_E_from_T(p->Tst[i], p->C[i], p->Lc[i], p->Ts[i], p->Tl[i]);
    }
}

void oracle_step(oracle_problem *p, int64_t n_steps, double dt)
{
    if (p->form == 1) {
        for (int64_t s = 0; s < n_steps; s++) {
            oracle_step_apparent(p, dt);
            p->step += 1;
            p->time += dt;
        }
        return;
    }
    for (int64_t s = 0; s < n_steps; s++) {
        oracle_temperatures(p, p->T);
        double qin = oracle_residual(p, p->T, p->R);
        p->Qb += dt * qin;
        for (int64_t i = 0; i < p->n_nodes; i++) {
            if (p->is_dir[i])
                p->E[i] = oracle_E_from_T(p->T_dir[i], p->C[i], p->Lc[i], p->Ts[i], p->Tl[i]);
            else
                p->E[i] += dt * p->R[i];
        }
        p->step += 1;
        p->time += dt;
    }
}

/* out = {U, U0, cumulative boundary heat, latent heat not yet released} */
void oracle_energy(const oracle_problem *p, double *out)
{
    double U = 0.0, lat = 0.0;
    for (int64_t i = 0; i < p->n_nodes; i++) {
        U += p->E[i];
        if (p->Lc[i] > 0.0) {
            double T = oracle_T_from_E(p->E[i], p->C[i], p->Lc[i], p->Ts[i], p->Tl[i]);
            double fl;
            if (p->Tl[i] <= p->Ts[i]) {
                /* isothermal: the liquid fraction is read off the plateau */
                fl = (p->E[i] - p->C[i] * T) / p->Lc[i];
                fl = fl < 0.0 ? 0.0 : (fl > 1.0 ? 1.0 : fl);
            } else {
                fl = oracle_liquid_fraction(T, p->Ts[i], p->Tl[i]);
            }
            lat += p->Lc[i] * fl;
        }
    }
    out[0] = U; out[1] = p->U0; out[2] = p->Qb; out[3] = lat;
}

/* ------------------------------------------------------------------------ */
/* Stable time step (reading of Eq. 13)                                      */
/* ------------------------------------------------------------------------ */

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* dt = 2 / max_i (sum_j |K_ij| + sum_j |H_ij|) / C_i over non-Dirichlet
 * nodes, with K the assembled conductance and H the assembled Robin face
 * matrix: a Gershgorin bound on the largest eigenvalue of C^{-1}(K + H),
 * which makes the explicit update of the linear (sensible-only) problem
 * stable.  The assembled row of node i is formed by collecting, over the
 * elements and faces that contain i, the pairs (j, entry) and summing equal j. */
double oracle_stable_dt(const oracle_problem *p)
{
    int64_t N = p->n_nodes;
    int64_t *cnt = calloc((size_t)N + 1, sizeof(int64_t));
    for (int64_t e = 0; e < p->n_tets; e++)
        for (int a = 0; a < 4; a++) cnt[p->tets[4 * e + a] + 1] += 4;
    for (int64_t f = 0; f < p->n_faces; f++)
        for (int a = 0; a < 3; a++) cnt[p->faces[3 * f + a] + 1] += 3;
    for (int64_t f = 0; f < p->n_if; f++)
        for (int a = 0; a < 3; a++) cnt[p->if_faces[3 * f + a] + 1] += 6;
    for (int64_t i = 0; i < N; i++) cnt[i + 1] += cnt[i];
    int64_t total = cnt[N];
    int32_t *col = malloc((size_t)total * sizeof(int32_t));
    double *val = malloc((size_t)total * sizeof(double));
    int64_t *fill = malloc((size_t)N * sizeof(int64_t));
    for (int64_t i = 0; i < N; i++) fill[i] = cnt[i];
    for (int64_t e = 0; e < p->n_tets; e++)
        for (int a = 0; a < 4; a++) {
            int32_t i = p->tets[4 * e + a];
            /* with a k(T) table the largest k of the table bounds K^e(T) */
            int32_t mt = p->emat[e];
            double kmax = 0.0;
            for (int32_t j = 0; j < p->kt_n[mt]; j++)
                if (p->kt_k[ORACLE_KT_MAX * mt + j] > kmax) kmax = p->kt_k[ORACLE_KT_MAX * mt + j];
            for (int b = 0; b < 4; b++) {
                col[fill[i]] = p->tets[4 * e + b];
                val[fill[i]] = p->kt_n[mt] > 0 ? kmax * p->Kg[16 * e + 4 * a + b]
                                               : p->Ke[16 * e + 4 * a + b];
                fill[i]++;
            }
        }
    for (int64_t f = 0; f < p->n_faces; f++) {
        double hA12 = p->fh[f] * p->farea[f] / 12.0;
        for (int a = 0; a < 3; a++) {
            int32_t i = p->faces[3 * f + a];
            for (int b = 0; b < 3; b++) {
                col[fill[i]] = p->faces[3 * f + b];
                val[fill[i]] = hA12 * (a == b ? 2.0 : 1.0);
                fill[i]++;
            }
        }
    }
    /* interface faces: the face matrix h A/12 (1 + delta) and the coupling
     * to the sister's nodes, -h A/9 per (face node, sister node) pair */
    for (int64_t f = 0; f < p->n_if; f++) {
        double hA12 = p->if_h[f] * p->if_area[f] / 12.0, hA9 = p->if_h[f] * p->if_area[f] / 9.0;
        const int32_t *sn = p->if_faces + 3 * p->if_sister[f];
        for (int a = 0; a < 3; a++) {
            int32_t i = p->if_faces[3 * f + a];
            for (int b = 0; b < 3; b++) {
                col[fill[i]] = p->if_faces[3 * f + b];
                val[fill[i]] = hA12 * (a == b ? 2.0 : 1.0);
                fill[i]++;
                col[fill[i]] = sn[b];
                val[fill[i]] = -hA9;
                fill[i]++;
            }
        }
    }
    double lam = 0.0;
    int32_t *idx = NULL; size_t idx_cap = 0;
    for (int64_t i = 0; i < N; i++) {
        int64_t b = cnt[i], n = cnt[i + 1] - cnt[i];
        if (n == 0 || p->is_dir[i]) continue;
        /* sort the row's column ids, keeping values alongside via a
         * position permutation */
        if ((size_t)n > idx_cap) { idx_cap = (size_t)n; idx = realloc(idx, idx_cap * 2 * sizeof(int32_t)); }
        /* pack (col, position) pairs and sort by col (stable enough: sums) */
        for (int64_t k = 0; k < n; k++) { idx[2 * k] = col[b + k]; idx[2 * k + 1] = (int32_t)k; }
        qsort(idx, (size_t)n, 2 * sizeof(int32_t), cmp_i32);
        double row = 0.0;
        int64_t k = 0;
        while (k < n) {
            int32_t j = idx[2 * k];
            double s = 0.0;
            while (k < n && idx[2 * k] == j) { s += val[b + idx[2 * k + 1]]; k++; }
            row += fabs(s);
        }
        double r = row / p->C[i];
        if (r > lam) lam = r;
    }
    free(idx); free(fill); free(val); free(col); free(cnt);
    return lam > 0.0 ? 2.0 / lam : INFINITY;
}

/* ------------------------------------------------------------------------ */
/* Accessors                                                                 */
/* ------------------------------------------------------------------------ */

int64_t oracle_n_nodes(const oracle_problem *p) { return p->n_nodes; }
int64_t oracle_step_count(const oracle_problem *p) { return p->step; }
double oracle_time(const oracle_problem *p) { return p->time; }

void oracle_get_E(const oracle_problem *p, double *out)
{
    memcpy(out, p->E, (size_t)p->n_nodes * sizeof(double));
}

void oracle_set_E(oracle_problem *p, const double *E)
{
    memcpy(p->E, E, (size_t)p->n_nodes * sizeof(double));
    for (int64_t i = 0; i < p->n_nodes; i++)
        p->Tst[i] = oracle_T_from_E(p->E[i], p->C[i], p->Lc[i], p->Ts[i], p->Tl[i]);
}

void oracle_get_lumped(const oracle_problem *p, double *C, double *m, double *Lc)
{
    memcpy(C, p->C, (size_t)p->n_nodes * sizeof(double));
    memcpy(m, p->m, (size_t)p->n_nodes * sizeof(double));
    memcpy(Lc, p->Lc, (size_t)p->n_nodes * sizeof(double));
}

void oracle_get_element(const oracle_problem *p, int64_t e, int32_t *nodes, double *K, double *vol)
{
    memcpy(nodes, p->tets + 4 * e, 4 * sizeof(int32_t));
    memcpy(K, p->Ke + 16 * e, 16 * sizeof(double));
    *vol = p->vol[e];
}
