/*
 * FP64 CPU oracle for the TensorMD energy / force / virial evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow definition that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header, table or
 * constant with the CUDA library; it is compiled by gcc with
 * -O2 -ffp-contract=off so that every floating-point expression is evaluated
 * exactly as written (no fused multiply-add).
 *
 * Paper: "TensorMD: Scalable Tensor-Diagram based Machine Learning Interatomic
 * Potential on Heterogeneous Many-Core Processors" (arXiv 2310.08439).
 * Each function names the section / equation it follows.  Readings of points
 * the paper leaves open:
 *   - D_ij = x_j + s*L - x_i (s = periodic image), R = |D|, Dhat = D/R
 *     (Sec. "The Tensor Formalism", the R_abc / D_abcx definitions; the printed
 *     formula there is garbled, this is the reading consistent with the
 *     r^alpha / r^m factors of the TensorMD descriptor equation).
 *   - f_k(r) = exp(-eta (r - mu)^2), f_c(r) = (cos(pi r / rc) + 1) / 2 for
 *     r < rc and 0 otherwise; h_k = f_k f_c  (the paper allows any f_k).
 *   - pair type b = species of the neighbour; the centre species selects the
 *     network and the (centre, neighbour) radial parameters.
 *   - sigma for m = 0 is sqrt, so G_k0 = |P_k0|; its derivative uses
 *     sign(P) with sign(0) = 0.
 *   - g_ij = dE/dD_ij; F_i += g_ij, F_j -= g_ij ("ScatterSum");
 *     virial W_ab = -sum_pairs D^a g^b (strain derivative of -E).
 *   - pairs with R >= rc contribute nothing (strict r^2 < rc^2 in FP64).
 * Parity pins for every function here live in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Model description (plain data, filled from Python through ctypes).        */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t S;          /* number of species                                 */
    int32_t K;          /* number of radial channels                         */
    int32_t L;          /* number of hidden layers                           */
    int32_t act;        /* 0 = tanh, 1 = SquarePlus                          */
    double rc;          /* cutoff radius (A)                                 */
    double sp_b;        /* SquarePlus b                                      */
    const double *mu;   /* [S][S][K]                                         */
    const double *eta;  /* [S][S][K]                                         */
    const int32_t *widths;      /* [L] hidden widths                         */
    const double *const *w;     /* [S] flat weights: per layer W[out][in], b */
    int32_t tab_ppa;    /* 0: H evaluated directly; > 0: tabulated H with    */
                        /* this many grid points per Angstrom (see below)    */
    int32_t tab_n;      /* grid points of tab_H / tab_dH per species pair     */
    const double *tab_H;   /* NULL: grid values from the Gaussians; else the  */
    const double *tab_dH;  /* caller's H, H' [S][S][tab_n][K] at R_g = g/ppa  */
} tmdo_model;

#define NMOM 20
#define MMAX 4

/* ------------------------------------------------------------------------- */
/* Moment tensor M_d and multiplicity T_dm  (Eq. T_dm, Sec. Tensor Formalism) */
/* Row order of T_dm:  1 | x y z | xx xy xz yy yz zz |                       */
/*                     xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz               */
/* Each row is the monomial ux^a uy^b uz^c with the exponents below; T is the */
/* number of distinct orderings of that monomial's Cartesian indices.        */
/* ------------------------------------------------------------------------- */
static const int MOM_EXP[NMOM][3] = {
    {0, 0, 0},
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
    {2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2},
    {3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1}, {1, 0, 2},
    {0, 3, 0}, {0, 2, 1}, {0, 1, 2}, {0, 0, 3}};

static const double T_DM[NMOM][MMAX] = {
    {1, 0, 0, 0},
    {0, 1, 0, 0}, {0, 1, 0, 0}, {0, 1, 0, 0},
    {0, 0, 1, 0}, {0, 0, 2, 0}, {0, 0, 2, 0}, {0, 0, 1, 0}, {0, 0, 2, 0}, {0, 0, 1, 0},
    {0, 0, 0, 1}, {0, 0, 0, 3}, {0, 0, 0, 3}, {0, 0, 0, 3}, {0, 0, 0, 6},
    {0, 0, 0, 3}, {0, 0, 0, 1}, {0, 0, 0, 3}, {0, 0, 0, 3}, {0, 0, 0, 1}};

static double ipow(double x, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r = r * x;
    return r;
}

static int rank_of(int d) { return MOM_EXP[d][0] + MOM_EXP[d][1] + MOM_EXP[d][2]; }

/* M_d(u) for a unit vector u. */
void tmdo_moments(const double *u, double *M) {
    for (int d = 0; d < NMOM; ++d)
        M[d] = ipow(u[0], MOM_EXP[d][0]) * ipow(u[1], MOM_EXP[d][1]) * ipow(u[2], MOM_EXP[d][2]);
}

/* dM_d/du_y (treating the three components as independent), [20][3]. */
void tmdo_moment_grad(const double *u, double *dM) {
    for (int d = 0; d < NMOM; ++d) {
        for (int y = 0; y < 3; ++y) {
            int e[3] = {MOM_EXP[d][0], MOM_EXP[d][1], MOM_EXP[d][2]};
            if (e[y] == 0) { dM[d * 3 + y] = 0.0; continue; }
            double c = (double)e[y];
            e[y] -= 1;
            dM[d * 3 + y] = c * ipow(u[0], e[0]) * ipow(u[1], e[1]) * ipow(u[2], e[2]);
        }
    }
}

void tmdo_tdm(double *T) { memcpy(T, T_DM, sizeof(T_DM)); }

/* ------------------------------------------------------------------------- */
/* Radial tensor H_k = f_k(r) f_c(r) and dH_k/dr   (Sec. Tensor Formalism,   */
/* the definition of H_abck from h^(k) = f_k f_c)                            */
/* ------------------------------------------------------------------------- */
static void radial_direct(const tmdo_model *m, int ti, int tj, double r, double *H, double *dH) {
    const int K = m->K;
    const double rc = m->rc;
    double fc = 0.0, dfc = 0.0;
    if (r < rc) {
        fc = 0.5 * (cos(M_PI * r / rc) + 1.0);
        dfc = -0.5 * (M_PI / rc) * sin(M_PI * r / rc);
    }
    for (int k = 0; k < K; ++k) {
        const double mu = m->mu[((size_t)ti * m->S + tj) * K + k];
        const double eta = m->eta[((size_t)ti * m->S + tj) * K + k];
        const double fk = exp(-eta * (r - mu) * (r - mu));
        const double dfk = -2.0 * eta * (r - mu) * fk;
        H[k] = fk * fc;
        dH[k] = dfk * fc + fk * dfc;
    }
}

/* ------------------------------------------------------------------------- */
/* Cubic Hermite interpolation on [x0, x0 + h] from the end values y0, y1 and */
/* slopes d0, d1, at x = x0 + t h (textbook basis h00 = 2t^3 - 3t^2 + 1,      */
/* h10 = t^3 - 2t^2 + t, h01 = -2t^3 + 3t^2, h11 = t^3 - t^2).  Exact for     */
/* cubic polynomials; error O(h^4) in y and O(h^3) in dy/dx.                  */
/* ------------------------------------------------------------------------- */
void tmdo_hermite(double y0, double d0, double y1, double d1, double h, double t, double *y, double *dy) {
    const double t2 = t * t, t3 = t2 * t;
    *y = (2.0 * t3 - 3.0 * t2 + 1.0) * y0 + (t3 - 2.0 * t2 + t) * h * d0
       + (-2.0 * t3 + 3.0 * t2) * y1 + (t3 - t2) * h * d1;
    *dy = ((6.0 * t2 - 6.0 * t) * y0 + (3.0 * t2 - 4.0 * t + 1.0) * h * d0
         + (-6.0 * t2 + 6.0 * t) * y1 + (3.0 * t2 - 2.0 * t) * h * d1) / h;
}

/* ------------------------------------------------------------------------- */
/* Tabulated radial tensor (Sec. "The H_abck tensor and Batch Rational 1D     */
/* Interpolation"): H and H' are read from a table of H_k(R_g), H'_k(R_g) on  */
/* the grid R_g = g / ppa, with the cutoff folded in (entries zero from rc    */
/* on), and interpolated between grid points.  The paper uses Kerley's        */
/* rational interpolation, whose formulas it does not print; this reading     */
/* interpolates the same table with cubic Hermite polynomials.  The grid      */
/* values are computed here directly in FP64 (the table is never stored).     */
/* ------------------------------------------------------------------------- */
static void radial_tab(const tmdo_model *m, int ti, int tj, double r, double *H, double *dH) {
    const int K = m->K;
    const double h = 1.0 / (double)m->tab_ppa;
    const double x = r * (double)m->tab_ppa;
    const double g = floor(x);
    const double t = x - g;
    double H0[256], dH0[256], H1[256], dH1[256];
    const double r0 = g * h, r1 = (g + 1.0) * h;
    if (m->tab_H) {   /* the caller's grid values; zero from rc on */
        const int gi = (int)g;
        for (int k = 0; k < K; ++k) {
            const size_t base = ((size_t)ti * m->S + tj) * (size_t)m->tab_n;
            const int ok0 = r0 < m->rc && gi < m->tab_n, ok1 = r1 < m->rc && gi + 1 < m->tab_n;
            H0[k] = ok0 ? m->tab_H[(base + gi) * K + k] : 0.0;
            dH0[k] = ok0 ? m->tab_dH[(base + gi) * K + k] : 0.0;
            H1[k] = ok1 ? m->tab_H[(base + gi + 1) * K + k] : 0.0;
            dH1[k] = ok1 ? m->tab_dH[(base + gi + 1) * K + k] : 0.0;
        }
    } else {
        radial_direct(m, ti, tj, r0, H0, dH0);   /* zero for r0 >= rc */
        radial_direct(m, ti, tj, r1, H1, dH1);
    }
    for (int k = 0; k < K; ++k) tmdo_hermite(H0[k], dH0[k], H1[k], dH1[k], h, t, &H[k], &dH[k]);
}

void tmdo_radial(const tmdo_model *m, int ti, int tj, double r, double *H, double *dH) {
    if (m->tab_ppa > 0 && r < m->rc)
        radial_tab(m, ti, tj, r, H, dH);
    else
        radial_direct(m, ti, tj, r, H, dH);
}

/* ------------------------------------------------------------------------- */
/* Neighbour set: every (j, s) with |x_j + s*L - x_i|^2 < r_list^2,           */
/* (j, s) != (i, 0).  Brute force over all j and all images s with           */
/* |s_x| <= ceil(r/L_x) + 1 on periodic axes (0 otherwise).  When every       */
/* periodic L_x > 2 r, at most one image per axis can be inside r and the    */
/* search uses the minimum image s_x = -rint((x_j - x_i)/L_x) only.           */
/* Output per atom is ordered by (j, sx, sy, sz).                            */
/* Sec. Tensor Formalism (R_abc, the neighbour table) and Sec. Evaluation    */
/* (binning with a buffer).                                                  */
/* ------------------------------------------------------------------------- */
static int in_range(const double *pos, const double *box, int i, int j,
                    int sx, int sy, int sz, double r2max) {
    const int s[3] = {sx, sy, sz};
    double d[3];
    for (int x = 0; x < 3; ++x) d[x] = (pos[3 * j + x] + (double)s[x] * box[x]) - pos[3 * i + x];
    const double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    return r2 < r2max;
}

/* Neighbours of atom i.  Writes at most cap entries; returns the count. */
int64_t tmdo_neighbors_of(int64_t n, const double *pos, const double *box, const int32_t *pbc,
                          double r_list, int64_t i, int64_t cap, int32_t *nbr, int8_t *shift) {
    const double r2max = r_list * r_list;
    int smax[3];
    int minimg = 1;
    for (int x = 0; x < 3; ++x) {
        smax[x] = pbc[x] ? (int)ceil(r_list / box[x]) + 1 : 0;
        if (pbc[x] && !(box[x] > 2.0 * r_list)) minimg = 0;
    }
    int64_t cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (minimg) {
            int s[3];
            for (int x = 0; x < 3; ++x)
                s[x] = pbc[x] ? -(int)rint((pos[3 * j + x] - pos[3 * i + x]) / box[x]) : 0;
            if (j == i && s[0] == 0 && s[1] == 0 && s[2] == 0) continue;
            if (in_range(pos, box, (int)i, (int)j, s[0], s[1], s[2], r2max)) {
                if (cnt < cap) {
                    nbr[cnt] = (int32_t)j;
                    for (int x = 0; x < 3; ++x) shift[3 * cnt + x] = (int8_t)s[x];
                }
                ++cnt;
            }
            continue;
        }
        for (int sx = -smax[0]; sx <= smax[0]; ++sx)
            for (int sy = -smax[1]; sy <= smax[1]; ++sy)
                for (int sz = -smax[2]; sz <= smax[2]; ++sz) {
                    if (j == i && sx == 0 && sy == 0 && sz == 0) continue;
                    if (!in_range(pos, box, (int)i, (int)j, sx, sy, sz, r2max)) continue;
                    if (cnt < cap) {
                        nbr[cnt] = (int32_t)j;
                        shift[3 * cnt + 0] = (int8_t)sx;
                        shift[3 * cnt + 1] = (int8_t)sy;
                        shift[3 * cnt + 2] = (int8_t)sz;
                    }
                    ++cnt;
                }
    }
    return cnt;
}

/* Full CSR list for all atoms.  counts[n] receives per-atom counts; when
 * off/nbr/shift are non-NULL they are filled (off must then hold n+1 and the
 * arrays sum(counts) entries).  Returns the total number of entries. */
int64_t tmdo_neighbors(int64_t n, const double *pos, const double *box, const int32_t *pbc,
                       double r_list, int64_t *counts, int64_t *off, int32_t *nbr, int8_t *shift) {
    if (off == NULL) {
        int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
        for (int64_t i = 0; i < n; ++i) {
            counts[i] = tmdo_neighbors_of(n, pos, box, pbc, r_list, i, 0, NULL, NULL);
            total += counts[i];
        }
        return total;
    }
    off[0] = 0;
    for (int64_t i = 0; i < n; ++i) off[i + 1] = off[i] + counts[i];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i)
        tmdo_neighbors_of(n, pos, box, pbc, r_list, i, counts[i], nbr + off[i], shift + 3 * off[i]);
    return off[n];
}

/* ------------------------------------------------------------------------- */
/* Atomic energy network (Sec. Tensor Formalism: E_a = NNP(G_abkm);          */
/* Sec. Evaluation: dense layers, SquarePlus or tanh).                       */
/* Forward through L hidden layers and a linear output; backward returns     */
/* dE_a/dG (standard back-propagation of the input gradient).                */
/* ------------------------------------------------------------------------- */
static double act_f(const tmdo_model *m, double z) {
    if (m->act == 0) return tanh(z);
    return 0.5 * (z + sqrt(z * z + m->sp_b));
}

static double act_df(const tmdo_model *m, double z) {
    if (m->act == 0) { const double t = tanh(z); return 1.0 - t * t; }
    return 0.5 * (1.0 + z / sqrt(z * z + m->sp_b));
}

#define MAXW 656

static double nnp(const tmdo_model *m, int s, const double *G, double *dEdG) {
    const int D = m->S * m->K * MMAX;
    int dims[8];
    dims[0] = D;
    for (int l = 0; l < m->L; ++l) dims[l + 1] = m->widths[l];
    dims[m->L + 1] = 1;
    const int nl = m->L + 1;
    double z[8][MAXW];   /* pre-activations of each layer */
    double a[9][MAXW];   /* a[0] = input, a[l+1] = act(z[l]) (output: identity) */
    const double *W[8], *b[8];
    const double *p = m->w[s];
    for (int l = 0; l < nl; ++l) {
        W[l] = p; p += (size_t)dims[l + 1] * dims[l];
        b[l] = p; p += dims[l + 1];
    }
    for (int c = 0; c < D; ++c) a[0][c] = G[c];
    for (int l = 0; l < nl; ++l) {
        for (int o = 0; o < dims[l + 1]; ++o) {
            double acc = b[l][o];
            for (int c = 0; c < dims[l]; ++c) acc += W[l][(size_t)o * dims[l] + c] * a[l][c];
            z[l][o] = acc;
            a[l + 1][o] = (l == nl - 1) ? acc : act_f(m, acc);
        }
    }
    const double E = a[nl][0];
    if (dEdG) {
        double g[MAXW], gn[MAXW];
        g[0] = 1.0; /* dE/dz of the linear output */
        for (int l = nl - 1; l >= 0; --l) {
            /* g = dE/dz[l]; propagate to dE/da[l] */
            for (int c = 0; c < dims[l]; ++c) {
                double acc = 0.0;
                for (int o = 0; o < dims[l + 1]; ++o) acc += W[l][(size_t)o * dims[l] + c] * g[o];
                gn[c] = acc;
            }
            if (l > 0)
                for (int c = 0; c < dims[l]; ++c) g[c] = gn[c] * act_df(m, z[l - 1][c]);
            else
                for (int c = 0; c < dims[0]; ++c) dEdG[c] = gn[c];
        }
    }
    return E;
}

/* ------------------------------------------------------------------------- */
/* Per-atom terms.  For centre atom a with neighbour entries (j, s):          */
/*   P_bkd  = sum_c H_bck M_bcd                          (P = M H)           */
/*   G_bkm  = sigma(sum_d T_dm P_bkd^2)                  (Eq. tensor_formalism, sigma_function) */
/*   E_a    = NNP(G)                                                          */
/*   P'_bkd = 2 T_dm sigma'_bkm P_bkd  * dE/dG_bkm       (Eq. dP_abkd)       */
/*   U_ck   = sum_d P'_bkd M_cd,  V_cd = sum_k P'_bkd H_ck   (Eq. U_abck)    */
/*   F1_cx  = sum_k U_ck H'_ck R'_cx,  F2_cx = sum_d V_cd M'_cxd             */
/*            (Eqs. F1_abcx, F2_abcx)                                         */
/* g[c] = F1_c + F2_c = dE_a/dD_c.  Returns E_a; G (Dd) and pair gradients   */
/* g (deg x 3) are written when non-NULL.                                    */
/* ------------------------------------------------------------------------- */
double tmdo_atom_terms(const tmdo_model *m, const double *pos, const int32_t *types,
                       const double *box, int64_t a, int64_t deg, const int32_t *nbr,
                       const int8_t *shift, double *G_out, double *g, double *dG_out) {
    const int S = m->S, K = m->K;
    const int D = S * K * MMAX;
    const int ti = types[a];
    const double rc2 = m->rc * m->rc;
    double *P = calloc((size_t)S * K * NMOM, sizeof(double));
    double *Pd = calloc((size_t)S * K * NMOM, sizeof(double));
    double *G = calloc((size_t)D, sizeof(double));
    double *dG = calloc((size_t)D, sizeof(double));
    double H[256], dH[256], M[NMOM], dM[NMOM * 3];

    /* setup (R, Dhat, H, M) and the contraction P = M H */
    for (int64_t c = 0; c < deg; ++c) {
        const int j = nbr[c];
        double Dv[3];
        for (int x = 0; x < 3; ++x)
            Dv[x] = (pos[3 * j + x] + (double)shift[3 * c + x] * box[x]) - pos[3 * a + x];
        const double r2 = (Dv[0] * Dv[0] + Dv[1] * Dv[1]) + Dv[2] * Dv[2];
        if (!(r2 < rc2)) continue;
        const double R = sqrt(r2);
        const double u[3] = {Dv[0] / R, Dv[1] / R, Dv[2] / R};
        const int b = types[j];
        tmdo_radial(m, ti, b, R, H, dH);
        tmdo_moments(u, M);
        for (int k = 0; k < K; ++k)
            for (int d = 0; d < NMOM; ++d) P[((size_t)b * K + k) * NMOM + d] += H[k] * M[d];
    }
    /* G_bkm = sigma(T_dm P^2) */
    for (int b = 0; b < S; ++b)
        for (int k = 0; k < K; ++k)
            for (int mm = 0; mm < MMAX; ++mm) {
                double s = 0.0;
                for (int d = 0; d < NMOM; ++d) {
                    const double p = P[((size_t)b * K + k) * NMOM + d];
                    s += T_DM[d][mm] * p * p;
                }
                G[((size_t)b * K + k) * MMAX + mm] = (mm == 0) ? sqrt(s) : s;
            }
    if (G_out) memcpy(G_out, G, sizeof(double) * D);
    const double Ea = nnp(m, ti, G, (g || dG_out) ? dG : NULL);
    if (dG_out) memcpy(dG_out, dG, sizeof(double) * D);
    if (g) {
        /* P' = 2 T sigma' P * dE/dG;  for m = 0: d|P|/dP = sign(P) */
        for (int b = 0; b < S; ++b)
            for (int k = 0; k < K; ++k)
                for (int d = 0; d < NMOM; ++d) {
                    const int mm = rank_of(d);
                    const double p = P[((size_t)b * K + k) * NMOM + d];
                    const double gg = dG[((size_t)b * K + k) * MMAX + mm];
                    double v;
                    if (mm == 0) v = gg * ((p > 0.0) ? 1.0 : ((p < 0.0) ? -1.0 : 0.0));
                    else v = 2.0 * T_DM[d][mm] * p * gg;
                    Pd[((size_t)b * K + k) * NMOM + d] = v;
                }
        for (int64_t c = 0; c < deg; ++c) {
            const int j = nbr[c];
            double Dv[3];
            for (int x = 0; x < 3; ++x)
                Dv[x] = (pos[3 * j + x] + (double)shift[3 * c + x] * box[x]) - pos[3 * a + x];
            const double r2 = (Dv[0] * Dv[0] + Dv[1] * Dv[1]) + Dv[2] * Dv[2];
            g[3 * c + 0] = g[3 * c + 1] = g[3 * c + 2] = 0.0;
            if (!(r2 < rc2)) continue;
            const double R = sqrt(r2);
            const double u[3] = {Dv[0] / R, Dv[1] / R, Dv[2] / R};
            const int b = types[j];
            tmdo_radial(m, ti, b, R, H, dH);
            tmdo_moments(u, M);
            tmdo_moment_grad(u, dM);
            const double *Pb = Pd + (size_t)b * K * NMOM;
            double U[256], V[NMOM];
            for (int k = 0; k < K; ++k) {
                double s = 0.0;
                for (int d = 0; d < NMOM; ++d) s += Pb[k * NMOM + d] * M[d];
                U[k] = s;
            }
            for (int d = 0; d < NMOM; ++d) {
                double s = 0.0;
                for (int k = 0; k < K; ++k) s += Pb[k * NMOM + d] * H[k];
                V[d] = s;
            }
            /* F1 = U H' R',  R'_x = dR/dD_x = u_x */
            double dEdR = 0.0;
            for (int k = 0; k < K; ++k) dEdR += U[k] * dH[k];
            /* F2 = V M', M'_xd = dM_d/dD_x = sum_y dM_d/du_y (delta_xy - u_x u_y)/R */
            double dEdu[3] = {0.0, 0.0, 0.0};
            for (int d = 0; d < NMOM; ++d)
                for (int y = 0; y < 3; ++y) dEdu[y] += V[d] * dM[d * 3 + y];
            const double udotg = u[0] * dEdu[0] + u[1] * dEdu[1] + u[2] * dEdu[2];
            for (int x = 0; x < 3; ++x)
                g[3 * c + x] = dEdR * u[x] + (dEdu[x] - u[x] * udotg) / R;
        }
    }
    free(P); free(Pd); free(G); free(dG);
    return Ea;
}

/* ------------------------------------------------------------------------- */
/* Whole-system evaluation: E, E_a, F_ax, virial (Sec. Tensor Formalism,     */
/* E = sum_a E_a, F_ax = -G' dG/dr_ax, F = ScatterSum(F1 + F2)).             */
/* forces / e_atom / virial / G / dG may be NULL; dG receives dE_a/dG_a.    */
/* ------------------------------------------------------------------------- */
int tmdo_compute(const tmdo_model *m, int64_t n, const double *pos, const int32_t *types,
                 const double *box, const int64_t *off, const int32_t *nbr, const int8_t *shift,
                 double *energy, double *e_atom, double *forces, double *virial, double *G,
                 double *dG) {
    const int D = m->S * m->K * MMAX;
    const int64_t nnz = off[n];
    double *g = (forces || virial) ? malloc(sizeof(double) * 3 * (size_t)(nnz > 0 ? nnz : 1)) : NULL;
    double *ea = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t a = 0; a < n; ++a)
        ea[a] = tmdo_atom_terms(m, pos, types, box, a, off[a + 1] - off[a], nbr + off[a],
                                shift + 3 * off[a], G ? G + (size_t)a * D : NULL,
                                g ? g + 3 * off[a] : NULL, dG ? dG + (size_t)a * D : NULL);
    double E = 0.0;
    for (int64_t a = 0; a < n; ++a) E += ea[a];
    if (energy) *energy = E;
    if (e_atom) memcpy(e_atom, ea, sizeof(double) * (size_t)n);
    if (forces) {
        memset(forces, 0, sizeof(double) * 3 * (size_t)n);
        for (int64_t a = 0; a < n; ++a)
            for (int64_t c = off[a]; c < off[a + 1]; ++c) {
                const int j = nbr[c];
                for (int x = 0; x < 3; ++x) {
                    forces[3 * a + x] += g[3 * c + x];
                    forces[3 * (size_t)j + x] -= g[3 * c + x];
                }
            }
    }
    if (virial) {
        double W[9] = {0};
        for (int64_t a = 0; a < n; ++a)
            for (int64_t c = off[a]; c < off[a + 1]; ++c) {
                const int j = nbr[c];
                double Dv[3];
                for (int x = 0; x < 3; ++x)
                    Dv[x] = (pos[3 * (size_t)j + x] + (double)shift[3 * c + x] * box[x]) - pos[3 * a + x];
                for (int al = 0; al < 3; ++al)
                    for (int be = 0; be < 3; ++be) W[al * 3 + be] -= Dv[al] * g[3 * c + be];
            }
        memcpy(virial, W, sizeof(W));
    }
    free(g); free(ea);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Velocity-Verlet step (Sec. Evaluation: 1 fs steps).  Units: A, fs, amu,  */
/* eV; a = F/m * CONV with CONV = 1/103.6427 (eV/(A amu) -> A/fs^2).         */
/* The caller supplies forces at the current positions and a callback-free  */
/* two-call protocol: vv_first (half kick + drift + wrap), then the caller   */
/* recomputes forces, then vv_second (half kick).                           */
/* ------------------------------------------------------------------------- */
#define CONV (1.0 / 103.6427)

void tmdo_vv_first(int64_t n, double *pos, double *vel, const double *forces, const double *mass,
                   const double *box, const int32_t *pbc, double dt) {
    for (int64_t i = 0; i < n; ++i)
        for (int x = 0; x < 3; ++x) {
            vel[3 * i + x] += 0.5 * dt * forces[3 * i + x] / mass[i] * CONV;
            double p = pos[3 * i + x] + dt * vel[3 * i + x];
            if (pbc[x]) {
                p = p - floor(p / box[x]) * box[x];
                if (p >= box[x]) p -= box[x];
                if (p < 0.0) p += box[x];
            }
            pos[3 * i + x] = p;
        }
}

void tmdo_vv_second(int64_t n, double *vel, const double *forces, const double *mass, double dt) {
    for (int64_t i = 0; i < n; ++i)
        for (int x = 0; x < 3; ++x) vel[3 * i + x] += 0.5 * dt * forces[3 * i + x] / mass[i] * CONV;
}

int tmdo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
