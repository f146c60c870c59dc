/*
 * pffrg_oracle.c -- plain, slow FP64 CPU oracle of the pf-FRG flow right-hand side.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is checked
 * against.  Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product library never does.  It shares no code, header,
 * table or constant generator with the CUDA path.
 *
 * What it computes (Buessen, "The SpinParser software for pseudofermion functional
 * renormalization group calculations on quantum magnets", arXiv:2109.13317):
 *   - Sec. 4.2, Eq. for omega_n: log frequency mesh; Sec. 5.2 cutoff mesh Lambda_n.
 *   - Sec. 3, Eq. (frg:parametrizationInitial): Sigma = 0, Gamma^{mu nu} = J^{mu nu}/4.
 *   - Sec. 3, Eqs. (frg:parametrizationBasis1p/2p): odd, imaginary Sigma; the
 *     frequency-sign, site-exchange and s<->u relations of Gamma.
 *   - Sec. 4.2: linear interpolation of Sigma, trilinear interpolation of Gamma with
 *     constant extrapolation; trapezoidal frequency integration on mesh nodes.
 *   - Sec. 3, Eqs. (frg:flowexplicit:1particle) and (frg:flowexplicit:2particle):
 *     the flow of Sigma (Hartree lattice sum + Fock on-site term) and of Gamma
 *     (s channel, t channel with the RPA lattice sum and two on-site terms, u channel)
 *     with the Katanin single-scale propagator; the spin sums alpha3, alpha4 are done
 *     literally on Pauli matrices (Eq. frg:parametrizationSpin) and projected back.
 *   - Sec. 4.3: Euler step Sigma(L - dL) = Sigma(L) - dL dSigma/dL (same for Gamma).
 *     An embedded Dormand-Prince 5(4) step is provided as well (not in the paper).
 *   - Sec. 3, Eq. (frg:correlation) and (frg:structurefactor): chi^{mu mu}_{ij}.
 *
 * Storage is translation-only: for every basis site b of the home cell, the vertex is
 * kept for every lattice site j within bond distance L of b (Sec. 4.1 truncation), with
 * no point-group reduction.  The first part keeps the spin-diagonal basis functions
 * Gamma^{cc}, c = 0..3 (the SU(2) and XYZ cores of Sec. 3); the section "General
 * time-reversal-invariant core" at the end keeps all 16 Gamma^{mu nu} as complex numbers
 * (the TRI core, any two-spin coupling).
 *
 * Readings of points the paper leaves open (same list as the design notes):
 *   C1  Sigma = -i gamma with gamma real and odd, so G(w) = 1/(i(w + gamma(w))).
 *   C2  each listed interaction S_from . M . S_to is one term of H; J_{ij} = M,
 *       J_{ji} = M^T.
 *   C3  theta(x) = 1 for x >= 0 in the delta-point terms; in the regular part the
 *       support of a trapezoid segment is tested at its midpoint and the integrand is
 *       evaluated without theta at both ends.
 *   C5  after mapping to s >= u, an interpolation corner (s_a, u_b) with s_a < u_b is
 *       read as -xi(nu) Gamma(u_b, t, s_a).
 *   C6  regular-part nodes: {+-w_n} and the propagator break points, clipped to
 *       [-w_max, w_max]; no tail beyond w_max.
 *   C7  arguments at 0 are non-negative (no site swap); gamma(0) = 0.
 *   C8  the bubble term of chi is local (delta_ij); the exchange part of the vertex
 *       term contributes only for i = j.
 *   C9  chi quadrature: exact integral of 1/(w+gamma(w))^2 per segment for piecewise
 *       linear gamma (plus an exact tail), product-trapezoid for the vertex term.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Frequency and cutoff meshes (Sec. 5.2)                                      */
/* ------------------------------------------------------------------------- */

/* omega_n = w_min (w_max / w_min)^(n / (N - 1)), n = 0..N-1. */
void or_mesh_exponential(int n, double wmin, double wmax, double* out) {
    for (int i = 0; i < n; ++i) {
        if (n == 1) { out[i] = wmin; continue; }
        out[i] = wmin * pow(wmax / wmin, (double)i / (double)(n - 1));
    }
}

/* Lambda_n = Lambda_max b^n for n = 0..floor(log_b(Lambda_min / Lambda_max)).
 * Returns the number of points; writes at most cap of them. */
int or_cutoff_exponential(double lmin, double lmax, double b, int cap, double* out) {
    int nmax = (int)floor(log(lmin / lmax) / log(b) + 1e-12);
    int cnt = nmax + 1;
    for (int i = 0; i < cnt && i < cap; ++i) out[i] = lmax * pow(b, (double)i);
    return cnt;
}

/* ------------------------------------------------------------------------- */
/* Pauli algebra: the spin sums of the flow equations, done literally           */
/* ------------------------------------------------------------------------- */

typedef struct { double re, im; } cx;
static cx cmul(cx a, cx b) { cx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static cx cadd(cx a, cx b) { cx r = {a.re + b.re, a.im + b.im}; return r; }

/* sigma^mu_{ab}: identity and the three Pauli matrices. */
static cx pauli(int mu, int a, int b) {
    cx z = {0.0, 0.0};
    switch (mu) {
    case 0: if (a == b) z.re = 1.0; break;
    case 1: if (a != b) z.re = 1.0; break;
    case 2: if (a == 0 && b == 1) z.im = -1.0; if (a == 1 && b == 0) z.im = 1.0; break;
    case 3: if (a == b) z.re = (a == 0) ? 1.0 : -1.0; break;
    }
    return z;
}

/* Spin tensor of a unit spin-diagonal basis function Gamma^{kk} = 1 (Eq. frg:parametrizationSpin):
 * V^{a b; c d} = sigma^k_{a c} sigma^k_{b d}. */
static cx unitV(int k, int a, int b, int c, int d) { return cmul(pauli(k, a, c), pauli(k, b, d)); }

/* Projection onto basis function (mu, nu): (1/4) sum sigma^mu_{1 1'} sigma^nu_{2 2'} T^{1' 2'; 1 2}. */
static cx project(int mu, int nu, cx T[2][2][2][2]) {
    cx acc = {0.0, 0.0};
    for (int a1p = 0; a1p < 2; ++a1p) for (int a2p = 0; a2p < 2; ++a2p)
    for (int a1 = 0; a1 < 2; ++a1) for (int a2 = 0; a2 < 2; ++a2)
        acc = cadd(acc, cmul(cmul(pauli(mu, a1, a1p), pauli(nu, a2, a2p)), T[a1p][a2p][a1][a2]));
    acc.re *= 0.25; acc.im *= 0.25;
    return acc;
}

/* Coefficient tables: out^{cc} += coef[term][c][k][l] A^{kk} B^{ll}.  Terms of Eq.
 * (frg:flowexplicit:2particle): 0 = s channel, 1 = t-channel lattice sum (without the
 * leading minus sign), 2 = t-channel first on-site term, 3 = second on-site term,
 * 4 = u channel. */
static double g_coef[5][4][4][4];
static double g_hartree[4], g_fock[4];      /* Sigma flow, Eq. (frg:flowexplicit:1particle) */
static double g_chi_dir[4][4], g_chi_exc[4][4]; /* chi vertex term, Eq. (frg:correlation) */
static int g_tables_ready = 0;
static int g_tables_closed = 1; /* 1 if every off-diagonal / imaginary projection vanished */

static void build_tables(void) {
    if (g_tables_ready) return;
    g_tables_closed = 1;
    for (int term = 0; term < 5; ++term)
    for (int k = 0; k < 4; ++k) for (int l = 0; l < 4; ++l) {
        cx T[2][2][2][2];
        for (int a1p = 0; a1p < 2; ++a1p) for (int a2p = 0; a2p < 2; ++a2p)
        for (int a1 = 0; a1 < 2; ++a1) for (int a2 = 0; a2 < 2; ++a2) {
            cx acc = {0.0, 0.0};
            for (int a3 = 0; a3 < 2; ++a3) for (int a4 = 0; a4 < 2; ++a4) {
                cx p;
                switch (term) {
                case 0: /* Gamma^{1'2';34} Gamma^{34;12} */
                    p = cmul(unitV(k, a1p, a2p, a3, a4), unitV(l, a3, a4, a1, a2)); break;
                case 1: /* Gamma^{1'4;13}_{i1 j} Gamma^{32';42}_{j i2} */
                    p = cmul(unitV(k, a1p, a4, a1, a3), unitV(l, a3, a2p, a4, a2)); break;
                case 2: /* Gamma^{1'4;13}_{i1 i2} Gamma^{2'3;42}_{i2 i2} */
                    p = cmul(unitV(k, a1p, a4, a1, a3), unitV(l, a2p, a3, a4, a2)); break;
                case 3: /* Gamma^{41';13}_{i1 i1} Gamma^{32';42}_{i1 i2} */
                    p = cmul(unitV(k, a4, a1p, a1, a3), unitV(l, a3, a2p, a4, a2)); break;
                default: /* Gamma^{42';13} Gamma^{1'3;42} */
                    p = cmul(unitV(k, a4, a2p, a1, a3), unitV(l, a1p, a3, a4, a2)); break;
                }
                acc = cadd(acc, p);
            }
            T[a1p][a2p][a1][a2] = acc;
        }
        for (int mu = 0; mu < 4; ++mu) for (int nu = 0; nu < 4; ++nu) {
            cx pr = project(mu, nu, T);
            if (mu == nu) {
                g_coef[term][mu][k][l] = pr.re;
                if (fabs(pr.im) > 1e-12) g_tables_closed = 0;
            } else if (fabs(pr.re) > 1e-12 || fabs(pr.im) > 1e-12) {
                g_tables_closed = 0;
            }
        }
    }
    /* Sigma flow: sum_{alpha2} Gamma^{a1 a2; a1 a2} (Hartree) and Gamma^{a2 a1; a1 a2} (Fock),
     * for alpha1 = up; alpha1 = down must give the same (checked). */
    for (int k = 0; k < 4; ++k) {
        for (int a1 = 0; a1 < 2; ++a1) {
            cx h = {0, 0}, f = {0, 0};
            for (int a2 = 0; a2 < 2; ++a2) {
                h = cadd(h, unitV(k, a1, a2, a1, a2));
                f = cadd(f, unitV(k, a2, a1, a1, a2));
            }
            if (a1 == 0) { g_hartree[k] = h.re; g_fock[k] = f.re; }
            else if (fabs(h.re - g_hartree[k]) > 1e-12 || fabs(f.re - g_fock[k]) > 1e-12) g_tables_closed = 0;
            if (fabs(h.im) > 1e-12 || fabs(f.im) > 1e-12) g_tables_closed = 0;
        }
    }
    /* chi vertex term: sum sigma^mu_{1 1'} sigma^mu_{2 2'} x (direct Gamma^{1'2';12},
     * exchanged Gamma^{2'1';12}). */
    for (int mu = 0; mu < 4; ++mu) for (int k = 0; k < 4; ++k) {
        cx d = {0, 0}, x = {0, 0};
        for (int a1p = 0; a1p < 2; ++a1p) for (int a2p = 0; a2p < 2; ++a2p)
        for (int a1 = 0; a1 < 2; ++a1) for (int a2 = 0; a2 < 2; ++a2) {
            cx pre = cmul(pauli(mu, a1, a1p), pauli(mu, a2, a2p));
            d = cadd(d, cmul(pre, unitV(k, a1p, a2p, a1, a2)));
            x = cadd(x, cmul(pre, unitV(k, a2p, a1p, a1, a2)));
        }
        g_chi_dir[mu][k] = d.re; g_chi_exc[mu][k] = x.re;
        if (fabs(d.im) > 1e-12 || fabs(x.im) > 1e-12) g_tables_closed = 0;
    }
    g_tables_ready = 1;
}

/* Export of the generated tables, for the pins that check them. */
int or_spin_tables(double* coef /*5*4*4*4*/, double* hartree, double* fock, double* chi_dir, double* chi_exc) {
    build_tables();
    memcpy(coef, g_coef, sizeof(g_coef));
    memcpy(hartree, g_hartree, sizeof(g_hartree));
    memcpy(fock, g_fock, sizeof(g_fock));
    memcpy(chi_dir, g_chi_dir, sizeof(g_chi_dir));
    memcpy(chi_exc, g_chi_exc, sizeof(g_chi_exc));
    return g_tables_closed;
}

/* ------------------------------------------------------------------------- */
/* Lattice: sites within bond distance L of each basis site (Sec. 4.1)           */
/* ------------------------------------------------------------------------- */

typedef struct { int n[3]; int b; } Site;

typedef struct {
    int nb;
    double prim[3][3];  /* prim[i] = a_i (Cartesian) */
    double* basis;      /* nb x 3 */
    int nbond;
    int* bonds;         /* nbond x 5: from, to, da0, da1, da2 */
    int L;
    int R;              /* bound on |n_i| of sites within range */
    int* nsite;         /* per basis b: number of sites within range */
    Site** sites;       /* per basis b: list */
    int** index;        /* per basis b: dense map (n+R, b') -> position in list or -1 */
    double** J;         /* per basis b: per site k: 3x3 coupling J_{b, k} */
    int offdiag;        /* 1 if some coupling has an off-diagonal entry */
} OrLattice;

static int dense_idx(const OrLattice* la, const int n[3], int b) {
    int W = 2 * la->R + 1;
    for (int i = 0; i < 3; ++i) if (n[i] < -la->R || n[i] > la->R) return -1;
    return (((n[0] + la->R) * W + (n[1] + la->R)) * W + (n[2] + la->R)) * la->nb + b;
}

/* Position of site k within range of basis b1 (home cell), or -1 if out of range. */
static int site_of(const OrLattice* la, int b1, const int d[3], int b2) {
    int di = dense_idx(la, d, b2);
    if (di < 0) return -1;
    return la->index[b1][di];
}

void or_lattice_free(OrLattice* la);

OrLattice* or_lattice_new(int nb, const double* prim, const double* basis, int nbond, const int* bonds,
                          int ncoup, const int* coup_from, const int* coup_to, const double* coup_M, int L) {
    if (nb <= 0 || L < 0) return NULL;
    OrLattice* la = (OrLattice*)calloc(1, sizeof(OrLattice));
    la->nb = nb; la->L = L; la->nbond = nbond;
    memcpy(la->prim, prim, 9 * sizeof(double));
    la->basis = (double*)malloc(sizeof(double) * 3 * nb);
    memcpy(la->basis, basis, sizeof(double) * 3 * nb);
    la->bonds = (int*)malloc(sizeof(int) * 5 * (nbond > 0 ? nbond : 1));
    memcpy(la->bonds, bonds, sizeof(int) * 5 * nbond);
    int maxda = 1;
    for (int e = 0; e < nbond; ++e) for (int i = 0; i < 3; ++i) {
        int a = abs(bonds[5 * e + 2 + i]); if (a > maxda) maxda = a;
    }
    la->R = L * maxda;
    int W = 2 * la->R + 1;
    size_t dense = (size_t)W * W * W * nb;
    la->nsite = (int*)calloc(nb, sizeof(int));
    la->sites = (Site**)calloc(nb, sizeof(Site*));
    la->index = (int**)calloc(nb, sizeof(int*));
    la->J = (double**)calloc(nb, sizeof(double*));
    for (int b = 0; b < nb; ++b) {
        /* breadth-first search over bonds from (0, b), depth L */
        int* idx = (int*)malloc(sizeof(int) * dense);
        for (size_t i = 0; i < dense; ++i) idx[i] = -1;
        int cap = 64, cnt = 0;
        Site* list = (Site*)malloc(sizeof(Site) * cap);
        int* depth = (int*)malloc(sizeof(int) * cap);
        Site s0 = {{0, 0, 0}, b};
        list[0] = s0; depth[0] = 0; cnt = 1;
        idx[dense_idx(la, s0.n, b)] = 0;
        for (int head = 0; head < cnt; ++head) {
            if (depth[head] >= L) continue;
            Site cur = list[head];
            for (int e = 0; e < nbond; ++e) {
                for (int dir = 0; dir < 2; ++dir) {
                    int from = bonds[5 * e], to = bonds[5 * e + 1];
                    Site nx;
                    if (dir == 0) {
                        if (cur.b != from) continue;
                        nx.b = to;
                        for (int i = 0; i < 3; ++i) nx.n[i] = cur.n[i] + bonds[5 * e + 2 + i];
                    } else {
                        if (cur.b != to) continue;
                        nx.b = from;
                        for (int i = 0; i < 3; ++i) nx.n[i] = cur.n[i] - bonds[5 * e + 2 + i];
                    }
                    int di = dense_idx(la, nx.n, nx.b);
                    if (di < 0 || idx[di] >= 0) continue;
                    if (cnt == cap) {
                        cap *= 2;
                        list = (Site*)realloc(list, sizeof(Site) * cap);
                        depth = (int*)realloc(depth, sizeof(int) * cap);
                    }
                    list[cnt] = nx; depth[cnt] = depth[head] + 1; idx[di] = cnt; ++cnt;
                }
            }
        }
        free(depth);
        la->nsite[b] = cnt; la->sites[b] = list; la->index[b] = idx;
        /* couplings J_{(0,b), k}: sum of M over listed interactions from (0,b) to k,
         * plus M^T over interactions from k to (0,b) (reading C2) */
        double* J = (double*)calloc((size_t)cnt * 9, sizeof(double));
        for (int c = 0; c < ncoup; ++c) {
            const int* f = coup_from + 4 * c; const int* t = coup_to + 4 * c;
            const double* M = coup_M + 9 * c;
            if (f[3] == b) {
                int d[3] = {t[0] - f[0], t[1] - f[1], t[2] - f[2]};
                int k = site_of(la, b, d, t[3]);
                if (k >= 0) for (int i = 0; i < 9; ++i) J[9 * k + i] += M[i];
            }
            if (t[3] == b) {
                int d[3] = {f[0] - t[0], f[1] - t[1], f[2] - t[2]};
                int k = site_of(la, b, d, f[3]);
                if (k >= 0) for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) J[9 * k + 3 * i + j] += M[3 * j + i];
            }
        }
        for (int k = 0; k < cnt; ++k) for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j)
            if (i != j && fabs(J[9 * k + 3 * i + j]) > 0.0) la->offdiag = 1;
        la->J[b] = J;
    }
    return la;
}

void or_lattice_free(OrLattice* la) {
    if (!la) return;
    for (int b = 0; b < la->nb; ++b) { free(la->sites[b]); free(la->index[b]); free(la->J[b]); }
    free(la->nsite); free(la->sites); free(la->index); free(la->J);
    free(la->basis); free(la->bonds); free(la);
}

int or_lattice_nsites(const OrLattice* la, int b) { return la->nsite[b]; }
int or_lattice_offdiag(const OrLattice* la) { return la->offdiag; }
/* out: n0, n1, n2, b' of site k within range of basis b. */
void or_lattice_site(const OrLattice* la, int b, int k, int* out) {
    Site s = la->sites[b][k];
    out[0] = s.n[0]; out[1] = s.n[1]; out[2] = s.n[2]; out[3] = s.b;
}
void or_lattice_coupling(const OrLattice* la, int b, int k, double* out9) { memcpy(out9, la->J[b] + 9 * k, 9 * sizeof(double)); }
/* -1 if (d, b2) is not within range of basis b1. */
int or_lattice_find(const OrLattice* la, int b1, const int* d, int b2) { return site_of(la, b1, d, b2); }

/* ------------------------------------------------------------------------- */
/* Vertex state                                                                */
/* ------------------------------------------------------------------------- */

typedef struct {
    const OrLattice* la;
    int N;            /* positive mesh frequencies */
    double* w;        /* mesh, ascending */
    int npair;        /* N(N+1)/2 pairs (s_i >= u_i) */
    size_t* off;      /* per basis b: offset of its block in G */
    size_t ntot;      /* total number of Gamma entries */
    double* gam;      /* gamma(w_n), Sigma = -i gamma */
    double* G;        /* Gamma^{cc}: [b][k][c][pair][t] */
    /* scratch for one right-hand side */
    double* dgam;
    double lam;       /* cutoff at which dgam was computed */
} OrState;

static size_t pair_index(int si, int ui) { return (size_t)si * (si + 1) / 2 + ui; }

static size_t g_index(const OrState* st, int b, int k, int c, int si, int ti, int ui) {
    return st->off[b] + ((((size_t)k * 4 + c) * st->npair + pair_index(si, ui)) * st->N + ti);
}

OrState* or_state_new(const OrLattice* la, int N, const double* mesh) {
    if (N < 2) return NULL;
    build_tables();
    OrState* st = (OrState*)calloc(1, sizeof(OrState));
    st->la = la; st->N = N;
    st->w = (double*)malloc(sizeof(double) * N);
    memcpy(st->w, mesh, sizeof(double) * N);
    st->npair = N * (N + 1) / 2;
    st->off = (size_t*)malloc(sizeof(size_t) * la->nb);
    size_t acc = 0;
    for (int b = 0; b < la->nb; ++b) { st->off[b] = acc; acc += (size_t)la->nsite[b] * 4 * st->npair * N; }
    st->ntot = acc;
    st->gam = (double*)calloc(N, sizeof(double));
    st->dgam = (double*)calloc(N, sizeof(double));
    st->G = (double*)calloc(acc, sizeof(double));
    return st;
}

void or_state_free(OrState* st) {
    if (!st) return;
    free(st->w); free(st->off); free(st->gam); free(st->dgam); free(st->G); free(st);
}

size_t or_state_size(const OrState* st) { return st->ntot; }
size_t or_state_offset(const OrState* st, int b) { return st->off[b]; }
void or_state_get(const OrState* st, double* gam, double* G) {
    if (gam) memcpy(gam, st->gam, sizeof(double) * st->N);
    if (G) memcpy(G, st->G, sizeof(double) * st->ntot);
}
void or_state_set(OrState* st, const double* gam, const double* G) {
    if (gam) memcpy(st->gam, gam, sizeof(double) * st->N);
    if (G) memcpy(st->G, G, sizeof(double) * st->ntot);
}

/* Initial condition, Eq. (frg:parametrizationInitial): gamma = 0, Gamma^{cc} = J^{cc}/4 for
 * c = x, y, z, Gamma^{00} = 0.  Frequency independent. */
void or_state_init(OrState* st) {
    memset(st->gam, 0, sizeof(double) * st->N);
    const OrLattice* la = st->la;
    for (int b = 0; b < la->nb; ++b)
    for (int k = 0; k < la->nsite[b]; ++k)
    for (int c = 0; c < 4; ++c) {
        double v = (c == 0) ? 0.0 : la->J[b][9 * k + 4 * (c - 1)] / 4.0;
        for (int p = 0; p < st->npair; ++p) for (int t = 0; t < st->N; ++t)
            st->G[st->off[b] + ((((size_t)k * 4 + c) * st->npair + p) * st->N + t)] = v;
    }
}

/* ------------------------------------------------------------------------- */
/* Interpolation (Sec. 4.2)                                                    */
/* ------------------------------------------------------------------------- */

/* Nearest lesser / greater mesh points of x >= 0 with the weights of the paper's linear
 * interpolation formula; constant extrapolation outside [w_0, w_{N-1}]. */
static void bracket(const double* w, int N, double x, int* lo, double* wlo, double* whi) {
    if (x <= w[0]) { *lo = 0; *wlo = 1.0; *whi = 0.0; return; }
    if (x >= w[N - 1]) { *lo = N - 2; *wlo = 0.0; *whi = 1.0; return; }
    int a = 0, b = N - 1; /* w[a] <= x < w[b] */
    while (b - a > 1) { int m = (a + b) / 2; if (w[m] <= x) a = m; else b = m; }
    *lo = a;
    *wlo = (w[a + 1] - x) / (w[a + 1] - w[a]);
    *whi = (x - w[a]) / (w[a + 1] - w[a]);
}

/* gamma(x): odd, linearly interpolated on |x| with constant extrapolation, gamma(0) = 0. */
static double interp_odd(const double* w, int N, const double* f, double x) {
    if (x == 0.0) return 0.0;
    double ax = fabs(x);
    int lo; double wl, wh;
    bracket(w, N, ax, &lo, &wl, &wh);
    double v = wl * f[lo] + wh * f[lo + 1];
    return x < 0 ? -v : v;
}

static double xi(int c) { return c == 0 ? 1.0 : -1.0; }

/* Stored value with the s <-> u exchange applied for corners below the diagonal (C5). */
static double stored(const OrState* st, int b, int k, int c, int si, int ti, int ui) {
    if (si >= ui) return st->G[g_index(st, b, k, c, si, ti, ui)];
    return -xi(c) * st->G[g_index(st, b, k, c, ui, ti, si)];
}

/* Gamma^{cc}_{i1 i2}(s, t, u) for i1 = (0, b1), i2 = (d, b2): symmetry relations
 * (frg:parametrizationBasis2p) to reach s, t, u >= 0 and s >= u, then trilinear
 * interpolation (Sec. 4.2).  Zero beyond the truncation range. */
static void lookup(const OrState* st, int b1, const int d[3], int b2, double s, double t, double u, double out[4]) {
    double fac[4] = {1.0, 1.0, 1.0, 1.0};
    int swap = 0;
    /* t -> -t: factor xi(mu) xi(nu) = 1 for spin-diagonal functions */
    if (t < 0) t = -t;
    /* s -> -s: exchange the sites (and mu <-> nu, a no-op on the diagonal) */
    if (s < 0) { s = -s; swap ^= 1; }
    /* u -> -u: factor xi xi = 1, exchange the sites */
    if (u < 0) { u = -u; swap ^= 1; }
    int ib = b1, jb = b2, dd[3] = {d[0], d[1], d[2]};
    if (swap) { ib = b2; jb = b1; dd[0] = -d[0]; dd[1] = -d[1]; dd[2] = -d[2]; }
    int k = site_of(st->la, ib, dd, jb);
    if (k < 0) { out[0] = out[1] = out[2] = out[3] = 0.0; return; }
    /* s < u: Gamma(s,t,u) = -xi(nu) Gamma(u,t,s) */
    if (s < u) {
        double tmp = s; s = u; u = tmp;
        for (int c = 0; c < 4; ++c) fac[c] = -xi(c);
    }
    int sl, tl, ul; double sw0, sw1, tw0, tw1, uw0, uw1;
    bracket(st->w, st->N, s, &sl, &sw0, &sw1);
    bracket(st->w, st->N, t, &tl, &tw0, &tw1);
    bracket(st->w, st->N, u, &ul, &uw0, &uw1);
    for (int c = 0; c < 4; ++c) {
        double v =
            uw0 * (tw0 * (sw0 * stored(st, ib, k, c, sl, tl, ul) + sw1 * stored(st, ib, k, c, sl + 1, tl, ul)) +
                   tw1 * (sw0 * stored(st, ib, k, c, sl, tl + 1, ul) + sw1 * stored(st, ib, k, c, sl + 1, tl + 1, ul))) +
            uw1 * (tw0 * (sw0 * stored(st, ib, k, c, sl, tl, ul + 1) + sw1 * stored(st, ib, k, c, sl + 1, tl, ul + 1)) +
                   tw1 * (sw0 * stored(st, ib, k, c, sl, tl + 1, ul + 1) + sw1 * stored(st, ib, k, c, sl + 1, tl + 1, ul + 1)));
        out[c] = fac[c] * v;
    }
}

void or_vertex_lookup(const OrState* st, int b1, const int* d, int b2, double s, double t, double u, double* out4) {
    lookup(st, b1, d, b2, s, t, u, out4);
}

/* ------------------------------------------------------------------------- */
/* Propagators (Sec. 3) with Sigma = -i gamma (C1)                              */
/* ------------------------------------------------------------------------- */

/* g(a) g(b) with g(x) = 1/(i (x + gamma(x))): real, -1 / ((a + gamma_a)(b + gamma_b)). */
static double prop_gg(const OrState* st, double a, double b) {
    double ga = a + interp_odd(st->w, st->N, st->gam, a);
    double gb = b + interp_odd(st->w, st->N, st->gam, b);
    return -1.0 / (ga * gb);
}

/* g(a) r(b) with the Katanin part r(x) = -g(x)^2 dSigma/dLambda(x):
 * real, -dgamma(b) / ((a + gamma_a)(b + gamma_b)^2). */
static double prop_gr(const OrState* st, double a, double b) {
    double ga = a + interp_odd(st->w, st->N, st->gam, a);
    double gb = b + interp_odd(st->w, st->N, st->gam, b);
    double db = interp_odd(st->w, st->N, st->dgam, b);
    return -db / (ga * gb * gb);
}

static double theta(double x) { return x >= 0.0 ? 1.0 : 0.0; }

enum { CH_S = 0, CH_T = 1, CH_U = 2 };

/* Regular (Katanin) propagator pair of a channel at integration frequency x, without theta. */
static double preg(const OrState* st, int ch, double v, double x) {
    switch (ch) {
    case CH_S: return prop_gr(st, x, v - x) + prop_gr(st, v - x, x);  /* G(w)S(s-w) + G(s-w)S(w) */
    case CH_T: return prop_gr(st, x, x - v) + prop_gr(st, x - v, x);  /* G(w)S(w-t) + G(w-t)S(w) */
    default:   return prop_gr(st, x, v + x) + prop_gr(st, v + x, x);  /* G(w)S(u+w) + G(u+w)S(w) */
    }
}

static int in_support(double lam, int ch, double v, double m) {
    if (fabs(m) < lam) return 0;
    switch (ch) {
    case CH_S: return fabs(v - m) >= lam;
    case CH_T: return fabs(m - v) >= lam;
    default:   return fabs(v + m) >= lam;
    }
}

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Integration nodes and weights of the w' integral of one channel at transfer frequency v:
 * four delta points of S (exact) and the trapezoidal rule on the regular Katanin part
 * (C3, C6).  Weights include the 1/(2 pi) prefactor.  Returns the node count. */
static int channel_nodes(const OrState* st, int ch, double v, double* x, double* W) {
    const double lam = st->lam;
    const double inv2pi = 1.0 / (2.0 * OR_PI);
    int n = 0;
    /* a delta point whose partner propagator G(a) lies below the cutoff (theta = 0) is absent:
     * the term is zero, not 0 * g(a), which diverges where a + gamma(a) = 0 */
    for (int sg = 0; sg < 2; ++sg) {
        double L = sg == 0 ? lam : -lam;
        double a, th;
        switch (ch) {
        case CH_S:  /* G(w) S(s - w): w = s - L;  G(s - w) S(w): w = L */
            a = v - L; th = theta(fabs(a) - lam);
            x[n] = a; W[n] = th != 0.0 ? prop_gg(st, a, L) * inv2pi : 0.0; ++n;
            x[n] = L; W[n] = th != 0.0 ? prop_gg(st, a, L) * inv2pi : 0.0; ++n;
            break;
        case CH_T:  /* G(w) S(w - t): w = t + L;  G(w - t) S(w): w = L */
            a = v + L; th = theta(fabs(a) - lam);
            x[n] = a; W[n] = th != 0.0 ? prop_gg(st, a, L) * inv2pi : 0.0; ++n;
            a = L - v; th = theta(fabs(a) - lam);
            x[n] = L; W[n] = th != 0.0 ? prop_gg(st, a, L) * inv2pi : 0.0; ++n;
            break;
        default:    /* G(w) S(u + w): w = L - u;  G(u + w) S(w): w = L */
            a = L - v; th = theta(fabs(a) - lam);
            x[n] = a; W[n] = th != 0.0 ? prop_gg(st, a, L) * inv2pi : 0.0; ++n;
            a = v + L; th = theta(fabs(a) - lam);
            x[n] = L; W[n] = th != 0.0 ? prop_gg(st, a, L) * inv2pi : 0.0; ++n;
            break;
        }
    }
    /* regular part: trapezoid on {+-w_n} and the break points, clipped to [-w_max, w_max] */
    int N = st->N, m = 0;
    double wmax = st->w[N - 1];
    double* pts = (double*)malloc(sizeof(double) * (2 * N + 4));
    for (int i = 0; i < N; ++i) { pts[m++] = st->w[i]; pts[m++] = -st->w[i]; }
    double bp[4];
    switch (ch) {
    case CH_S: bp[0] = lam; bp[1] = -lam; bp[2] = v + lam; bp[3] = v - lam; break;
    case CH_T: bp[0] = lam; bp[1] = -lam; bp[2] = v + lam; bp[3] = v - lam; break;
    default:   bp[0] = lam; bp[1] = -lam; bp[2] = -v + lam; bp[3] = -v - lam; break;
    }
    for (int i = 0; i < 4; ++i) {
        double q = bp[i];
        if (q > wmax) q = wmax;
        if (q < -wmax) q = -wmax;
        pts[m++] = q;
    }
    qsort(pts, m, sizeof(double), cmp_double);
    for (int i = 0; i < m; ++i) {
        double wgt = 0.0;
        if (i > 0 && pts[i] > pts[i - 1] && in_support(lam, ch, v, 0.5 * (pts[i] + pts[i - 1])))
            wgt += 0.5 * (pts[i] - pts[i - 1]);
        if (i + 1 < m && pts[i + 1] > pts[i] && in_support(lam, ch, v, 0.5 * (pts[i] + pts[i + 1])))
            wgt += 0.5 * (pts[i + 1] - pts[i]);
        if (wgt == 0.0) continue;
        x[n] = pts[i];
        W[n] = wgt * preg(st, ch, v, pts[i]) * inv2pi;
        ++n;
    }
    free(pts);
    return n;
}

/* ------------------------------------------------------------------------- */
/* Flow of the self-energy, Eq. (frg:flowexplicit:1particle)                    */
/* ------------------------------------------------------------------------- */

/* dgamma/dLambda at frequency w1 for reference basis site b:
 * dSigma(w1) = -(1/2pi) sum_{w2 = +-Lambda} [sum_j Gamma_{i1 j}(w1+w2, 0, w1-w2)
 *              - Gamma_{i1 i1}(w1+w2, w2-w1, 0)] g(w2)  (spin sums as tabulated),
 * and with Sigma = -i gamma, g(w2) = -i/(w2 + gamma(w2)):
 * dgamma(w1) = -(1/2pi) sum_{w2} H(w1, w2) / (w2 + gamma(w2)). */
static double sigma_rhs_at(const OrState* st, int b, double w1, double lam) {
    const OrLattice* la = st->la;
    double acc = 0.0;
    for (int sg = 0; sg < 2; ++sg) {
        double w2 = sg == 0 ? lam : -lam;
        double H = 0.0, v[4];
        for (int k = 0; k < la->nsite[b]; ++k) {
            Site j = la->sites[b][k];
            lookup(st, b, j.n, j.b, w1 + w2, 0.0, w1 - w2, v);
            for (int c = 0; c < 4; ++c) H += g_hartree[c] * v[c];
        }
        int z[3] = {0, 0, 0};
        lookup(st, b, z, b, w1 + w2, w2 - w1, 0.0, v);
        for (int c = 0; c < 4; ++c) H -= g_fock[c] * v[c];
        acc += H / (w2 + interp_odd(st->w, st->N, st->gam, w2));
    }
    return -acc / (2.0 * OR_PI);
}

double or_sigma_rhs_point(OrState* st, int b, double w1, double lam) { return sigma_rhs_at(st, b, w1, lam); }

/* ------------------------------------------------------------------------- */
/* Flow of the two-particle vertex, Eq. (frg:flowexplicit:2particle)            */
/* ------------------------------------------------------------------------- */

static void accum(double out[4], double W, int term, const double A[4], const double B[4], double sign) {
    for (int c = 0; c < 4; ++c) {
        double acc = 0.0;
        for (int k = 0; k < 4; ++k) for (int l = 0; l < 4; ++l) acc += g_coef[term][c][k][l] * A[k] * B[l];
        out[c] += sign * W * acc;
    }
}

/* dGamma^{cc}_{i1 i2}(s, t, u)/dLambda for i1 = (0, b1), i2 = (d2, b2), arbitrary s, t, u.
 * Requires st->dgam / st->lam to hold the self-energy flow at this cutoff. */
static void gamma_rhs_at(const OrState* st, int b1, const int d2[3], int b2, double s, double t, double u,
                         double* xs, double* Ws, double out[4]) {
    const OrLattice* la = st->la;
    double w1p = (s + t + u) / 2, w2p = (s - t - u) / 2, w1 = (s - t + u) / 2, w2 = (s + t - u) / 2;
    double A[4], B[4], C[4];
    int z[3] = {0, 0, 0};
    out[0] = out[1] = out[2] = out[3] = 0.0;
    /* s channel: [G(w)S(s-w) + G(s-w)S(w)] Gamma(s, w1'-w, w-w2') Gamma(s, w-w1, w-w2) */
    int n = channel_nodes(st, CH_S, s, xs, Ws);
    for (int q = 0; q < n; ++q) {
        double x = xs[q];
        lookup(st, b1, d2, b2, s, w1p - x, x - w2p, A);
        lookup(st, b1, d2, b2, s, x - w1, x - w2, B);
        accum(out, Ws[q], 0, A, B, 1.0);
    }
    /* t channel: [G(w)S(w-t) + G(w-t)S(w)] x [ -sum_j Gamma_{i1 j}(w1+w, t, w1'-w) Gamma_{j i2}(w+w2', t, w-w2)
     *   + Gamma_{i1 i2}(w1+w, t, w1'-w) Gamma_{i2 i2}(w2'+w, w2-w, -t)
     *   + Gamma_{i1 i1}(w1+w, w-w1', -t) Gamma_{i1 i2}(w+w2', t, w-w2) ] */
    n = channel_nodes(st, CH_T, t, xs, Ws);
    for (int q = 0; q < n; ++q) {
        double x = xs[q];
        /* lattice sum over j within range of both i1 and i2 (lookup is zero beyond range) */
        for (int k = 0; k < la->nsite[b1]; ++k) {
            Site j = la->sites[b1][k];
            int dj2[3] = {d2[0] - j.n[0], d2[1] - j.n[1], d2[2] - j.n[2]};
            if (site_of(la, j.b, dj2, b2) < 0) continue;
            lookup(st, b1, j.n, j.b, w1 + x, t, w1p - x, A);
            lookup(st, j.b, dj2, b2, x + w2p, t, x - w2, B);
            accum(out, Ws[q], 1, A, B, -1.0);
        }
        lookup(st, b1, d2, b2, w1 + x, t, w1p - x, A);
        lookup(st, b2, z, b2, w2p + x, w2 - x, -t, C);
        accum(out, Ws[q], 2, A, C, 1.0);
        lookup(st, b1, z, b1, w1 + x, x - w1p, -t, C);
        lookup(st, b1, d2, b2, x + w2p, t, x - w2, B);
        accum(out, Ws[q], 3, C, B, 1.0);
    }
    /* u channel: [G(w)S(u+w) + G(u+w)S(w)] Gamma(w1+w, w-w2', u) Gamma(w1'+w, w2-w, u) */
    n = channel_nodes(st, CH_U, u, xs, Ws);
    for (int q = 0; q < n; ++q) {
        double x = xs[q];
        lookup(st, b1, d2, b2, w1 + x, x - w2p, u, A);
        lookup(st, b1, d2, b2, w1p + x, w2 - x, u, B);
        accum(out, Ws[q], 4, A, B, 1.0);
    }
}

/* The state keeps one self-energy for all sites, which presumes that every basis site is
 * equivalent (Sec. 4.1: the vertex is stored relative to a reference site; the self-energy is
 * site-independent by the same symmetry).  The flow of Sigma is therefore evaluated at every
 * basis site; where the sites disagree beyond rounding the lattice has inequivalent sites, the
 * largest relative difference is recorded and dgamma is set to NaN, so that no result is
 * silently computed with basis site 0's self-energy. */
static double g_sigma_basis_spread = 0.0;   /* largest relative spread seen across basis sites */
#define OR_BASIS_TOL 1e-10

static double basis_spread(const double* ref, const double* other, int N) {
    double num = 0.0, den = 0.0;
    for (int i = 0; i < N; ++i) {
        if (fabs(other[i] - ref[i]) > num) num = fabs(other[i] - ref[i]);
        if (fabs(ref[i]) > den) den = fabs(ref[i]);
    }
    return num == 0.0 ? 0.0 : num / (den > 0.0 ? den : 1e-300);
}

static void compute_dgam(OrState* st, double lam) {
    st->lam = lam;
    for (int i = 0; i < st->N; ++i) st->dgam[i] = sigma_rhs_at(st, 0, st->w[i], lam);
    double* other = (double*)malloc(sizeof(double) * st->N);
    for (int b = 1; b < st->la->nb; ++b) {
        for (int i = 0; i < st->N; ++i) other[i] = sigma_rhs_at(st, b, st->w[i], lam);
        double d = basis_spread(st->dgam, other, st->N);
        if (d > g_sigma_basis_spread) g_sigma_basis_spread = d;
        if (d > OR_BASIS_TOL)
            for (int i = 0; i < st->N; ++i) st->dgam[i] = NAN;
    }
    free(other);
}

/* Largest relative spread of the self-energy flow across basis sites seen so far (reset by
 * or_sigma_basis_spread_reset). */
double or_sigma_basis_spread(void) { return g_sigma_basis_spread; }
void or_sigma_basis_spread_reset(void) { g_sigma_basis_spread = 0.0; }

/* Full right-hand side at cutoff lam: dgamma (N) and dGamma (state layout). */
void or_rhs(OrState* st, double lam, double* dgam, double* dG) {
    compute_dgam(st, lam);
    if (dgam) memcpy(dgam, st->dgam, sizeof(double) * st->N);
    const OrLattice* la = st->la;
    const int N = st->N;
    for (int b = 0; b < la->nb; ++b) {
        int ns = la->nsite[b];
        long total = (long)ns * st->npair * N;
        #pragma omp parallel
        {
            double* xs = (double*)malloc(sizeof(double) * (2 * N + 16));
            double* Ws = (double*)malloc(sizeof(double) * (2 * N + 16));
            #pragma omp for schedule(dynamic, 16)
            for (long e = 0; e < total; ++e) {
                int k = (int)(e / ((long)st->npair * N));
                long rem = e % ((long)st->npair * N);
                int p = (int)(rem / N), ti = (int)(rem % N);
                int si = 0; while ((size_t)(si + 1) * (si + 2) / 2 <= (size_t)p) ++si;
                int ui = p - si * (si + 1) / 2;
                Site j = la->sites[b][k];
                double out[4];
                gamma_rhs_at(st, b, j.n, j.b, st->w[si], st->w[ti], st->w[ui], xs, Ws, out);
                for (int c = 0; c < 4; ++c) dG[g_index(st, b, k, c, si, ti, ui)] = out[c];
            }
            free(xs); free(Ws);
        }
    }
}

/* Right-hand side of selected stored entries only: ent = n x (b, k, si, ti, ui); out = n x 4. */
void or_rhs_entries(OrState* st, double lam, int n, const int* ent, double* out) {
    compute_dgam(st, lam);
    const int N = st->N;
    #pragma omp parallel
    {
        double* xs = (double*)malloc(sizeof(double) * (2 * N + 16));
        double* Ws = (double*)malloc(sizeof(double) * (2 * N + 16));
        #pragma omp for schedule(dynamic, 1)
        for (int e = 0; e < n; ++e) {
            const int* q = ent + 5 * e;
            Site j = st->la->sites[q[0]][q[1]];
            gamma_rhs_at(st, q[0], j.n, j.b, st->w[q[2]], st->w[q[3]], st->w[q[4]], xs, Ws, out + 4 * e);
        }
        free(xs); free(Ws);
    }
}

/* Right-hand side at arbitrary (s, t, u) and site pair (0, b1), (d, b2): used for the
 * symmetry-relation invariants.  dgam must be current (or_rhs_prepare). */
void or_rhs_prepare(OrState* st, double lam, double* dgam) {
    compute_dgam(st, lam);
    if (dgam) memcpy(dgam, st->dgam, sizeof(double) * st->N);
}
void or_rhs_point(const OrState* st, int b1, const int* d, int b2, double s, double t, double u, double* out4) {
    double xs[512], Ws[512];
    if (2 * st->N + 16 > 512) { out4[0] = out4[1] = out4[2] = out4[3] = NAN; return; }
    gamma_rhs_at(st, b1, d, b2, s, t, u, xs, Ws, out4);
}

/* Nodes and weights of one channel (after or_rhs_prepare), for the quadrature pins. */
int or_channel_nodes(const OrState* st, int ch, double v, double* x, double* W) { return channel_nodes(st, ch, v, x, W); }

/* ------------------------------------------------------------------------- */
/* Cutoff stepping (Sec. 4.3)                                                  */
/* ------------------------------------------------------------------------- */

/* Euler: y(Lambda - dLambda) = y(Lambda) - dLambda dy/dLambda. */
void or_euler_step(OrState* st, double lam, double lam_next) {
    double dl = lam - lam_next;
    double* dg = (double*)malloc(sizeof(double) * st->N);
    double* dG = (double*)malloc(sizeof(double) * st->ntot);
    or_rhs(st, lam, dg, dG);
    for (int i = 0; i < st->N; ++i) st->gam[i] -= dl * dg[i];
    for (size_t i = 0; i < st->ntot; ++i) st->G[i] -= dl * dG[i];
    free(dg); free(dG);
}

/* Dormand-Prince 5(4) tableau (Dormand & Prince 1980). */
static const double DP_C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0},
    {1.0 / 5},
    {3.0 / 40, 9.0 / 40},
    {44.0 / 45, -56.0 / 15, 32.0 / 9},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656},
    {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
static const double DP_B5[7] = {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0.0};
static const double DP_B4[7] = {5179.0 / 57600, 0.0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};

/* Export of the tableau for the order-condition pin: c[7], a[7*6], b5[7], b4[7]. */
void or_dp54_tableau(double* c, double* a, double* b5, double* b4) {
    memcpy(c, DP_C, sizeof(DP_C)); memcpy(a, DP_A, sizeof(DP_A));
    memcpy(b5, DP_B5, sizeof(DP_B5)); memcpy(b4, DP_B4, sizeof(DP_B4));
}

/* Dormand-Prince 5(4) (Dormand & Prince 1980) step of size h = lam_next - lam (negative when
 * integrating toward small cutoff).  The state advances with the fifth-order solution; the
 * return value is the normwise scaled error max_i |e_i| / (atol + rtol max_i max(|y_i|, |y_new_i|)). */
double or_dp54_step(OrState* st, double lam, double lam_next, double rtol, double atol) {
    const double h = lam_next - lam;
    const int N = st->N;
    const size_t M = st->ntot;
    double* y0g = (double*)malloc(sizeof(double) * N);
    double* y0G = (double*)malloc(sizeof(double) * M);
    memcpy(y0g, st->gam, sizeof(double) * N);
    memcpy(y0G, st->G, sizeof(double) * M);
    double* kg[7]; double* kG[7];
    for (int i = 0; i < 7; ++i) { kg[i] = (double*)malloc(sizeof(double) * N); kG[i] = (double*)malloc(sizeof(double) * M); }
    for (int s = 0; s < 7; ++s) {
        for (int i = 0; i < N; ++i) {
            double acc = 0.0;
            for (int r = 0; r < s; ++r) acc += DP_A[s][r] * kg[r][i];
            st->gam[i] = y0g[i] + h * acc;
        }
        for (size_t i = 0; i < M; ++i) {
            double acc = 0.0;
            for (int r = 0; r < s; ++r) acc += DP_A[s][r] * kG[r][i];
            st->G[i] = y0G[i] + h * acc;
        }
        or_rhs(st, lam + DP_C[s] * h, kg[s], kG[s]);
    }
    /* normwise scaled error: max_i |h (y5_i - y4_i)| / (atol + rtol max_i max(|y0_i|, |y5_i|)) */
    double emax = 0.0, ymax = 0.0;
    for (int i = 0; i < N; ++i) {
        double y5 = 0.0, y4 = 0.0;
        for (int r = 0; r < 7; ++r) { y5 += DP_B5[r] * kg[r][i]; y4 += DP_B4[r] * kg[r][i]; }
        double yn = y0g[i] + h * y5;
        emax = fmax(emax, fabs(h * (y5 - y4)));
        ymax = fmax(ymax, fmax(fabs(y0g[i]), fabs(yn)));
        st->gam[i] = yn;
    }
    for (size_t i = 0; i < M; ++i) {
        double y5 = 0.0, y4 = 0.0;
        for (int r = 0; r < 7; ++r) { y5 += DP_B5[r] * kG[r][i]; y4 += DP_B4[r] * kG[r][i]; }
        double yn = y0G[i] + h * y5;
        emax = fmax(emax, fabs(h * (y5 - y4)));
        ymax = fmax(ymax, fmax(fabs(y0G[i]), fabs(yn)));
        st->G[i] = yn;
    }
    double err = emax / (atol + rtol * ymax);
    for (int i = 0; i < 7; ++i) { free(kg[i]); free(kG[i]); }
    free(y0g); free(y0G);
    return err;
}

/* ------------------------------------------------------------------------- */
/* Correlations, Eq. (frg:correlation)                                         */
/* ------------------------------------------------------------------------- */

/* chi^{mu mu}_{b, k} for every basis site b and site k within its range:
 * out[(off_b + k) * 4 + mu] where off_b = sum of site counts of the lower basis sites.
 * Nodes: Lambda and the mesh points above it; segment weights are the exact integral of
 * 1/(w + gamma(w))^2 for piecewise-linear gamma, plus an exact tail beyond the last node
 * with gamma held constant (C9). */
void or_chi(const OrState* st, double lam, double* out) {
    const OrLattice* la = st->la;
    const int N = st->N;
    double* y = (double*)malloc(sizeof(double) * (N + 1));
    double* Wn = (double*)calloc(N + 1, sizeof(double));
    int K = 0;
    y[K++] = lam;
    for (int i = 0; i < N; ++i) if (st->w[i] > lam) y[K++] = st->w[i];
    for (int k = 0; k + 1 < K; ++k) {
        double ya = y[k] + interp_odd(st->w, N, st->gam, y[k]);
        double yb = y[k + 1] + interp_odd(st->w, N, st->gam, y[k + 1]);
        double seg = (y[k + 1] - y[k]) / (ya * yb);
        Wn[k] += 0.5 * seg; Wn[k + 1] += 0.5 * seg;
    }
    Wn[K - 1] += 1.0 / (y[K - 1] + interp_odd(st->w, N, st->gam, y[K - 1]));
    double bubble = 0.0;
    for (int k = 0; k < K; ++k) bubble += Wn[k];
    bubble /= (2.0 * OR_PI);
    /* symmetric node list: +-y_k with equal weights */
    int M = 2 * K;
    double* xs = (double*)malloc(sizeof(double) * M);
    double* ws = (double*)malloc(sizeof(double) * M);
    for (int k = 0; k < K; ++k) { xs[k] = y[k]; ws[k] = Wn[k]; xs[K + k] = -y[k]; ws[K + k] = Wn[k]; }
    size_t base = 0;
    for (int b = 0; b < la->nb; ++b) {
        int ns = la->nsite[b];
        #pragma omp parallel for schedule(dynamic, 1)
        for (int k = 0; k < ns; ++k) {
            Site j = la->sites[b][k];
            int onsite = (j.b == b && j.n[0] == 0 && j.n[1] == 0 && j.n[2] == 0);
            int z[3] = {0, 0, 0};
            double acc[4] = {0, 0, 0, 0};
            for (int p = 0; p < M; ++p) for (int q = 0; q < M; ++q) {
                double v[4], e[4];
                lookup(st, b, j.n, j.b, xs[p] + xs[q], 0.0, xs[p] - xs[q], v);
                if (onsite) lookup(st, b, z, b, xs[p] + xs[q], xs[q] - xs[p], 0.0, e);
                for (int mu = 0; mu < 4; ++mu) {
                    double F = 0.0;
                    for (int c = 0; c < 4; ++c) {
                        F += g_chi_dir[mu][c] * v[c];
                        if (onsite) F -= g_chi_exc[mu][c] * e[c];
                    }
                    acc[mu] += ws[p] * ws[q] * F;
                }
            }
            for (int mu = 0; mu < 4; ++mu)
                out[(base + k) * 4 + mu] = (onsite ? bubble : 0.0) - acc[mu] / (16.0 * OR_PI * OR_PI);
        }
        base += ns;
    }
    free(y); free(Wn); free(xs); free(ws);
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
void or_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ========================================================================= */
/* General time-reversal-invariant core: all 16 basis functions Gamma^{mu nu} */
/* ========================================================================= */
/*
 * The TRI core of Sec. 3 keeps every basis function Gamma^{mu nu}, mu, nu = 0..3, of the
 * parametrization Eq. (frg:parametrization), so that couplings with off-diagonal entries
 * (Dzyaloshinskii-Moriya, symmetric off-diagonal exchange) can be represented.  Here the
 * vertex is stored as complex numbers: the real / imaginary classes of Eq.
 * (frg:parametrizationBasis2p) are then a property the flow has to preserve, not an
 * assumption of the storage.  The spin sums alpha3, alpha4 are again done literally on
 * Pauli matrices and projected back (generalising build_tables to unit basis functions
 * Gamma^{kl} with k != l).  Same lattice (translation-only storage), meshes, propagators,
 * node sets and readings C1-C9 as the spin-diagonal oracle above; additional reading:
 *   C15 the self-energy flow takes the spin trace of Eq. (frg:flowexplicit:1particle)
 *       (the average over alpha1): by time-reversal invariance Sigma is spin-diagonal and
 *       alpha-independent, so the alpha1-odd part vanishes for a state of the right classes.
 * Layout: [b][k][mu * 4 + nu][pair(s,u)][t], complex.
 */

static cx cscale(cx a, double s) { cx r = {a.re * s, a.im * s}; return r; }

/* Spin tensor of a unit basis function Gamma^{kl} = 1: V^{a b; c d} = sigma^k_{a c} sigma^l_{b d}. */
static cx unitV2(int k, int l, int a, int b, int c, int d) { return cmul(pauli(k, a, c), pauli(l, b, d)); }

/* Non-zero projected coefficients of one term, out^{o} += coef A^{x} B^{y}. */
typedef struct { int o, x, y; cx coef; } TriCoef;
static TriCoef* g_tlist[5];
static int g_tcount[5];
static cx g_thart[16], g_tfock[16];              /* Sigma flow, averaged over alpha1 (C15) */
static cx g_tchi_dir[16][16], g_tchi_exc[16][16]; /* chi^{mu nu} vertex term */
static int g_ttables_ready = 0;

static void build_tri_tables(void) {
    if (g_ttables_ready) return;
    for (int term = 0; term < 5; ++term) {
        g_tlist[term] = (TriCoef*)malloc(sizeof(TriCoef) * 16 * 16 * 16);
        g_tcount[term] = 0;
        for (int x = 0; x < 16; ++x) for (int y = 0; y < 16; ++y) {
            const int k1 = x / 4, k2 = x % 4, l1 = y / 4, l2 = y % 4;
            cx T[2][2][2][2];
            for (int a1p = 0; a1p < 2; ++a1p) for (int a2p = 0; a2p < 2; ++a2p)
            for (int a1 = 0; a1 < 2; ++a1) for (int a2 = 0; a2 < 2; ++a2) {
                cx acc = {0.0, 0.0};
                for (int a3 = 0; a3 < 2; ++a3) for (int a4 = 0; a4 < 2; ++a4) {
                    cx p;
                    switch (term) {
                    case 0: /* Gamma^{1'2';34} Gamma^{34;12} */
                        p = cmul(unitV2(k1, k2, a1p, a2p, a3, a4), unitV2(l1, l2, a3, a4, a1, a2)); break;
                    case 1: /* Gamma^{1'4;13}_{i1 j} Gamma^{32';42}_{j i2} */
                        p = cmul(unitV2(k1, k2, a1p, a4, a1, a3), unitV2(l1, l2, a3, a2p, a4, a2)); break;
                    case 2: /* Gamma^{1'4;13}_{i1 i2} Gamma^{2'3;42}_{i2 i2} */
                        p = cmul(unitV2(k1, k2, a1p, a4, a1, a3), unitV2(l1, l2, a2p, a3, a4, a2)); break;
                    case 3: /* Gamma^{41';13}_{i1 i1} Gamma^{32';42}_{i1 i2} */
                        p = cmul(unitV2(k1, k2, a4, a1p, a1, a3), unitV2(l1, l2, a3, a2p, a4, a2)); break;
                    default: /* Gamma^{42';13} Gamma^{1'3;42} */
                        p = cmul(unitV2(k1, k2, a4, a2p, a1, a3), unitV2(l1, l2, a1p, a3, a4, a2)); break;
                    }
                    acc = cadd(acc, p);
                }
                T[a1p][a2p][a1][a2] = acc;
            }
            for (int o = 0; o < 16; ++o) {
                cx pr = project(o / 4, o % 4, T);
                if (fabs(pr.re) > 1e-12 || fabs(pr.im) > 1e-12) {
                    TriCoef c = {o, x, y, pr};
                    g_tlist[term][g_tcount[term]++] = c;
                }
            }
        }
    }
    for (int x = 0; x < 16; ++x) {
        const int k = x / 4, l = x % 4;
        cx h = {0, 0}, f = {0, 0};
        for (int a1 = 0; a1 < 2; ++a1) for (int a2 = 0; a2 < 2; ++a2) {
            h = cadd(h, unitV2(k, l, a1, a2, a1, a2));
            f = cadd(f, unitV2(k, l, a2, a1, a1, a2));
        }
        g_thart[x] = cscale(h, 0.5);
        g_tfock[x] = cscale(f, 0.5);
    }
    for (int o = 0; o < 16; ++o) for (int x = 0; x < 16; ++x) {
        const int mu = o / 4, nu = o % 4, k = x / 4, l = x % 4;
        cx d = {0, 0}, e = {0, 0};
        for (int a1p = 0; a1p < 2; ++a1p) for (int a2p = 0; a2p < 2; ++a2p)
        for (int a1 = 0; a1 < 2; ++a1) for (int a2 = 0; a2 < 2; ++a2) {
            cx pre = cmul(pauli(mu, a1, a1p), pauli(nu, a2, a2p));
            d = cadd(d, cmul(pre, unitV2(k, l, a1p, a2p, a1, a2)));
            e = cadd(e, cmul(pre, unitV2(k, l, a2p, a1p, a1, a2)));
        }
        g_tchi_dir[o][x] = d;
        g_tchi_exc[o][x] = e;
    }
    g_ttables_ready = 1;
}

/* Export of the generated TRI tables (dense, complex as re/im pairs): coef[5][16][16][16][2],
 * hartree[16][2], fock[16][2], chi_dir[16][16][2], chi_exc[16][16][2]. */
void or_tri_spin_tables(double* coef, double* hartree, double* fock, double* chi_dir, double* chi_exc) {
    build_tri_tables();
    memset(coef, 0, sizeof(double) * 5 * 4096 * 2);
    for (int term = 0; term < 5; ++term)
        for (int i = 0; i < g_tcount[term]; ++i) {
            const TriCoef* c = &g_tlist[term][i];
            size_t at = (((size_t)term * 16 + c->o) * 16 + c->x) * 16 + c->y;
            coef[2 * at] = c->coef.re; coef[2 * at + 1] = c->coef.im;
        }
    for (int x = 0; x < 16; ++x) {
        hartree[2 * x] = g_thart[x].re; hartree[2 * x + 1] = g_thart[x].im;
        fock[2 * x] = g_tfock[x].re; fock[2 * x + 1] = g_tfock[x].im;
    }
    for (int o = 0; o < 16; ++o) for (int x = 0; x < 16; ++x) {
        chi_dir[2 * (o * 16 + x)] = g_tchi_dir[o][x].re; chi_dir[2 * (o * 16 + x) + 1] = g_tchi_dir[o][x].im;
        chi_exc[2 * (o * 16 + x)] = g_tchi_exc[o][x].re; chi_exc[2 * (o * 16 + x) + 1] = g_tchi_exc[o][x].im;
    }
}

typedef struct {
    OrState f;     /* mesh, gamma, dgamma, cutoff of the self-energy flow (f.G unused) */
    size_t* off;   /* per basis b: offset of its block */
    size_t ntot;   /* complex entries */
    cx* G;
} OrStateT;

static size_t gT_index(const OrStateT* st, int b, int k, int c, int si, int ti, int ui) {
    return st->off[b] + ((((size_t)k * 16 + c) * st->f.npair + pair_index(si, ui)) * st->f.N + ti);
}

OrStateT* or_tri_state_new(const OrLattice* la, int N, const double* mesh) {
    if (N < 2) return NULL;
    build_tri_tables();
    OrStateT* st = (OrStateT*)calloc(1, sizeof(OrStateT));
    st->f.la = la; st->f.N = N;
    st->f.w = (double*)malloc(sizeof(double) * N);
    memcpy(st->f.w, mesh, sizeof(double) * N);
    st->f.npair = N * (N + 1) / 2;
    st->f.gam = (double*)calloc(N, sizeof(double));
    st->f.dgam = (double*)calloc(N, sizeof(double));
    st->off = (size_t*)malloc(sizeof(size_t) * la->nb);
    size_t acc = 0;
    for (int b = 0; b < la->nb; ++b) { st->off[b] = acc; acc += (size_t)la->nsite[b] * 16 * st->f.npair * N; }
    st->ntot = acc;
    st->G = (cx*)calloc(acc, sizeof(cx));
    return st;
}

void or_tri_state_free(OrStateT* st) {
    if (!st) return;
    free(st->f.w); free(st->f.gam); free(st->f.dgam); free(st->off); free(st->G); free(st);
}

size_t or_tri_state_size(const OrStateT* st) { return st->ntot; }
size_t or_tri_state_offset(const OrStateT* st, int b) { return st->off[b]; }
/* G as interleaved (re, im) pairs. */
void or_tri_state_get(const OrStateT* st, double* gam, double* G) {
    if (gam) memcpy(gam, st->f.gam, sizeof(double) * st->f.N);
    if (G) memcpy(G, st->G, sizeof(cx) * st->ntot);
}
void or_tri_state_set(OrStateT* st, const double* gam, const double* G) {
    if (gam) memcpy(st->f.gam, gam, sizeof(double) * st->f.N);
    if (G) memcpy(st->G, G, sizeof(cx) * st->ntot);
}

/* Eq. (frg:parametrizationInitial): gamma = 0, Gamma^{mu nu} = J^{mu nu}/4 for mu, nu = x, y, z,
 * every basis function with mu = 0 or nu = 0 zero.  Frequency independent, real. */
void or_tri_state_init(OrStateT* st) {
    const OrLattice* la = st->f.la;
    memset(st->f.gam, 0, sizeof(double) * st->f.N);
    for (int b = 0; b < la->nb; ++b)
    for (int k = 0; k < la->nsite[b]; ++k)
    for (int c = 0; c < 16; ++c) {
        const int mu = c / 4, nu = c % 4;
        cx v = {0.0, 0.0};
        if (mu > 0 && nu > 0) v.re = la->J[b][9 * k + 3 * (mu - 1) + (nu - 1)] / 4.0;
        for (int p = 0; p < st->f.npair; ++p) for (int t = 0; t < st->f.N; ++t)
            st->G[st->off[b] + (((size_t)k * 16 + c) * st->f.npair + p) * st->f.N + t] = v;
    }
}

/* Stored value of component (mu, nu) with the s <-> u exchange for corners below the
 * diagonal (C5): factor -xi(nu). */
static cx storedT(const OrStateT* st, int b, int k, int mu, int nu, int si, int ti, int ui) {
    if (si >= ui) return st->G[gT_index(st, b, k, 4 * mu + nu, si, ti, ui)];
    return cscale(st->G[gT_index(st, b, k, 4 * mu + nu, ui, ti, si)], -xi(nu));
}

/* Gamma^{mu nu}_{i1 i2}(s, t, u), all 16 components, for i1 = (0, b1), i2 = (d, b2): the
 * relations of Eq. (frg:parametrizationBasis2p) applied in the paper's order --
 *   t -> -t: factor xi(mu) xi(nu);
 *   s -> -s: exchange the sites and mu <-> nu;
 *   u -> -u: factor xi(mu) xi(nu), exchange the sites and mu <-> nu;
 *   s < u:   factor -xi(nu) with (s, u) exchanged --
 * then trilinear interpolation (Sec. 4.2).  Zero beyond the truncation range. */
static void lookupT(const OrStateT* st, int b1, const int d[3], int b2, double s, double t, double u, cx out[16]) {
    const double s0 = s, t0 = t, u0 = u;
    for (int c = 0; c < 16; ++c) {
        int m = c / 4, n = c % 4, swap = 0, tmp;
        double fac = 1.0;
        s = s0; t = t0; u = u0;
        if (t < 0) { t = -t; fac *= xi(m) * xi(n); }
        if (s < 0) { s = -s; swap ^= 1; tmp = m; m = n; n = tmp; }
        if (u < 0) { u = -u; fac *= xi(m) * xi(n); swap ^= 1; tmp = m; m = n; n = tmp; }
        int ib = b1, jb = b2, dd[3] = {d[0], d[1], d[2]};
        if (swap) { ib = b2; jb = b1; dd[0] = -d[0]; dd[1] = -d[1]; dd[2] = -d[2]; }
        int k = site_of(st->f.la, ib, dd, jb);
        if (k < 0) { out[c].re = out[c].im = 0.0; continue; }
        if (s < u) { double q = s; s = u; u = q; fac *= -xi(n); }
        int sl, tl, ul; double sw0, sw1, tw0, tw1, uw0, uw1;
        bracket(st->f.w, st->f.N, s, &sl, &sw0, &sw1);
        bracket(st->f.w, st->f.N, t, &tl, &tw0, &tw1);
        bracket(st->f.w, st->f.N, u, &ul, &uw0, &uw1);
        cx v = {0.0, 0.0};
        const double ws[2] = {sw0, sw1}, wt[2] = {tw0, tw1}, wu[2] = {uw0, uw1};
        for (int a = 0; a < 2; ++a) for (int bb = 0; bb < 2; ++bb) for (int e = 0; e < 2; ++e) {
            double wgt = ws[a] * wt[bb] * wu[e];
            if (wgt == 0.0) continue;
            v = cadd(v, cscale(storedT(st, ib, k, m, n, sl + a, tl + bb, ul + e), wgt));
        }
        out[c] = cscale(v, fac);
    }
}

void or_tri_lookup(const OrStateT* st, int b1, const int* d, int b2, double s, double t, double u, double* out32) {
    lookupT(st, b1, d, b2, s, t, u, (cx*)out32);
}

/* Self-energy flow with the spin trace (C15):
 * dgamma(w1) = -(1/2pi) sum_{w2 = +-Lambda} Re H(w1, w2) / (w2 + gamma(w2)),
 * H = sum_j h_x Gamma^x_{i1 j}(w1+w2, 0, w1-w2) - f_x Gamma^x_{i1 i1}(w1+w2, w2-w1, 0). */
static double g_tri_sigma_imag = 0.0;   /* largest |Im H| seen (zero for a state of the right classes) */
static double sigma_rhs_atT(const OrStateT* st, int b, double w1, double lam) {
    const OrLattice* la = st->f.la;
    double acc = 0.0;
    cx v[16];
    for (int sg = 0; sg < 2; ++sg) {
        double w2 = sg == 0 ? lam : -lam;
        cx H = {0.0, 0.0};
        for (int k = 0; k < la->nsite[b]; ++k) {
            Site j = la->sites[b][k];
            lookupT(st, b, j.n, j.b, w1 + w2, 0.0, w1 - w2, v);
            for (int x = 0; x < 16; ++x) H = cadd(H, cmul(g_thart[x], v[x]));
        }
        int z[3] = {0, 0, 0};
        lookupT(st, b, z, b, w1 + w2, w2 - w1, 0.0, v);
        for (int x = 0; x < 16; ++x) H = cadd(H, cscale(cmul(g_tfock[x], v[x]), -1.0));
        if (fabs(H.im) > g_tri_sigma_imag) g_tri_sigma_imag = fabs(H.im);
        acc += H.re / (w2 + interp_odd(st->f.w, st->f.N, st->f.gam, w2));
    }
    return -acc / (2.0 * OR_PI);
}

double or_tri_sigma_imag(void) { return g_tri_sigma_imag; }

static void accumT(cx out[16], double W, int term, const cx A[16], const cx B[16], double sign) {
    for (int i = 0; i < g_tcount[term]; ++i) {
        const TriCoef* c = &g_tlist[term][i];
        out[c->o] = cadd(out[c->o], cscale(cmul(c->coef, cmul(A[c->x], B[c->y])), sign * W));
    }
}

/* dGamma^{mu nu}_{i1 i2}(s, t, u)/dLambda, Eq. (frg:flowexplicit:2particle), as gamma_rhs_at
 * with all 16 components. */
static void gamma_rhs_atT(const OrStateT* st, int b1, const int d2[3], int b2, double s, double t, double u,
                          double* xs, double* Ws, cx out[16]) {
    const OrLattice* la = st->f.la;
    double w1p = (s + t + u) / 2, w2p = (s - t - u) / 2, w1 = (s - t + u) / 2, w2 = (s + t - u) / 2;
    cx A[16], B[16], C[16];
    int z[3] = {0, 0, 0};
    for (int c = 0; c < 16; ++c) out[c].re = out[c].im = 0.0;
    int n = channel_nodes(&st->f, CH_S, s, xs, Ws);
    for (int q = 0; q < n; ++q) {
        double x = xs[q];
        lookupT(st, b1, d2, b2, s, w1p - x, x - w2p, A);
        lookupT(st, b1, d2, b2, s, x - w1, x - w2, B);
        accumT(out, Ws[q], 0, A, B, 1.0);
    }
    n = channel_nodes(&st->f, CH_T, t, xs, Ws);
    for (int q = 0; q < n; ++q) {
        double x = xs[q];
        for (int k = 0; k < la->nsite[b1]; ++k) {
            Site j = la->sites[b1][k];
            int dj2[3] = {d2[0] - j.n[0], d2[1] - j.n[1], d2[2] - j.n[2]};
            if (site_of(la, j.b, dj2, b2) < 0) continue;
            lookupT(st, b1, j.n, j.b, w1 + x, t, w1p - x, A);
            lookupT(st, j.b, dj2, b2, x + w2p, t, x - w2, B);
            accumT(out, Ws[q], 1, A, B, -1.0);
        }
        lookupT(st, b1, d2, b2, w1 + x, t, w1p - x, A);
        lookupT(st, b2, z, b2, w2p + x, w2 - x, -t, C);
        accumT(out, Ws[q], 2, A, C, 1.0);
        lookupT(st, b1, z, b1, w1 + x, x - w1p, -t, C);
        lookupT(st, b1, d2, b2, x + w2p, t, x - w2, B);
        accumT(out, Ws[q], 3, C, B, 1.0);
    }
    n = channel_nodes(&st->f, CH_U, u, xs, Ws);
    for (int q = 0; q < n; ++q) {
        double x = xs[q];
        lookupT(st, b1, d2, b2, w1 + x, x - w2p, u, A);
        lookupT(st, b1, d2, b2, w1p + x, w2 - x, u, B);
        accumT(out, Ws[q], 4, A, B, 1.0);
    }
}

/* As compute_dgam: the self-energy flow at every basis site, NaN if they disagree. */
static void compute_dgamT(OrStateT* st, double lam) {
    st->f.lam = lam;
    for (int i = 0; i < st->f.N; ++i) st->f.dgam[i] = sigma_rhs_atT(st, 0, st->f.w[i], lam);
    double* other = (double*)malloc(sizeof(double) * st->f.N);
    for (int b = 1; b < st->f.la->nb; ++b) {
        for (int i = 0; i < st->f.N; ++i) other[i] = sigma_rhs_atT(st, b, st->f.w[i], lam);
        double d = basis_spread(st->f.dgam, other, st->f.N);
        if (d > g_sigma_basis_spread) g_sigma_basis_spread = d;
        if (d > OR_BASIS_TOL)
            for (int i = 0; i < st->f.N; ++i) st->f.dgam[i] = NAN;
    }
    free(other);
}

/* Full right-hand side: dgamma (N) and dGamma (state layout, interleaved re / im). */
void or_tri_rhs(OrStateT* st, double lam, double* dgam, double* dG) {
    compute_dgamT(st, lam);
    if (dgam) memcpy(dgam, st->f.dgam, sizeof(double) * st->f.N);
    const OrLattice* la = st->f.la;
    const int N = st->f.N, npair = st->f.npair;
    cx* out = (cx*)dG;
    for (int b = 0; b < la->nb; ++b) {
        long total = (long)la->nsite[b] * npair * N;
        #pragma omp parallel
        {
            double* xs = (double*)malloc(sizeof(double) * (2 * N + 16));
            double* Ws = (double*)malloc(sizeof(double) * (2 * N + 16));
            #pragma omp for schedule(dynamic, 4)
            for (long e = 0; e < total; ++e) {
                int k = (int)(e / ((long)npair * N));
                long rem = e % ((long)npair * N);
                int p = (int)(rem / N), ti = (int)(rem % N);
                int si = 0; while ((si + 1) * (si + 2) / 2 <= p) ++si;
                int ui = p - si * (si + 1) / 2;
                Site j = la->sites[b][k];
                cx o[16];
                gamma_rhs_atT(st, b, j.n, j.b, st->f.w[si], st->f.w[ti], st->f.w[ui], xs, Ws, o);
                for (int c = 0; c < 16; ++c) out[gT_index(st, b, k, c, si, ti, ui)] = o[c];
            }
            free(xs); free(Ws);
        }
    }
}

void or_tri_rhs_prepare(OrStateT* st, double lam, double* dgam) {
    compute_dgamT(st, lam);
    if (dgam) memcpy(dgam, st->f.dgam, sizeof(double) * st->f.N);
}
/* Right-hand side at an arbitrary (s, t, u) and site pair after or_tri_rhs_prepare:
 * out32 = 16 complex values. */
void or_tri_rhs_point(const OrStateT* st, int b1, const int* d, int b2, double s, double t, double u, double* out32) {
    double xs[512], Ws[512];
    if (2 * st->f.N + 16 > 512) { for (int i = 0; i < 32; ++i) out32[i] = NAN; return; }
    gamma_rhs_atT(st, b1, d, b2, s, t, u, xs, Ws, (cx*)out32);
}

/* Right-hand side of selected stored entries only (after or_tri_rhs_prepare):
 * ent = n x (b, k, si, ti, ui); out = n x 16 complex (interleaved). */
void or_tri_rhs_entries(const OrStateT* st, int n, const int* ent, double* out) {
    const int N = st->f.N;
    #pragma omp parallel
    {
        double* xs = (double*)malloc(sizeof(double) * (2 * N + 16));
        double* Ws = (double*)malloc(sizeof(double) * (2 * N + 16));
        #pragma omp for schedule(dynamic, 1)
        for (int e = 0; e < n; ++e) {
            const int* q = ent + 5 * e;
            Site j = st->f.la->sites[q[0]][q[1]];
            gamma_rhs_atT(st, q[0], j.n, j.b, st->f.w[q[2]], st->f.w[q[3]], st->f.w[q[4]], xs, Ws, (cx*)(out + 32 * (size_t)e));
        }
        free(xs); free(Ws);
    }
}

/* Euler step (Sec. 4.3). */
void or_tri_euler_step(OrStateT* st, double lam, double lam_next) {
    double dl = lam - lam_next;
    double* dg = (double*)malloc(sizeof(double) * st->f.N);
    double* dG = (double*)malloc(sizeof(cx) * st->ntot);
    or_tri_rhs(st, lam, dg, dG);
    for (int i = 0; i < st->f.N; ++i) st->f.gam[i] -= dl * dg[i];
    double* G = (double*)st->G;
    for (size_t i = 0; i < 2 * st->ntot; ++i) G[i] -= dl * dG[i];
    free(dg); free(dG);
}

/* Dormand-Prince 5(4) step of the TRI state (same tableau, stage sums and normwise error as
 * or_dp54_step; the complex vertex enters the norm through its real and imaginary parts). */
double or_tri_dp54_step(OrStateT* st, double lam, double lam_next, double rtol, double atol) {
    const double h = lam_next - lam;
    const int N = st->f.N;
    const size_t M = 2 * st->ntot;
    double* G = (double*)st->G;
    double* y0g = (double*)malloc(sizeof(double) * N);
    double* y0G = (double*)malloc(sizeof(double) * M);
    memcpy(y0g, st->f.gam, sizeof(double) * N);
    memcpy(y0G, G, sizeof(double) * M);
    double* kg[7]; double* kG[7];
    for (int i = 0; i < 7; ++i) { kg[i] = (double*)malloc(sizeof(double) * N); kG[i] = (double*)malloc(sizeof(double) * M); }
    for (int s = 0; s < 7; ++s) {
        for (int i = 0; i < N; ++i) {
            double acc = 0.0;
            for (int r = 0; r < s; ++r) acc += DP_A[s][r] * kg[r][i];
            st->f.gam[i] = y0g[i] + h * acc;
        }
        for (size_t i = 0; i < M; ++i) {
            double acc = 0.0;
            for (int r = 0; r < s; ++r) acc += DP_A[s][r] * kG[r][i];
            G[i] = y0G[i] + h * acc;
        }
        or_tri_rhs(st, lam + DP_C[s] * h, kg[s], kG[s]);
    }
    double emax = 0.0, ymax = 0.0;
    for (int i = 0; i < N; ++i) {
        double y5 = 0.0, y4 = 0.0;
        for (int r = 0; r < 7; ++r) { y5 += DP_B5[r] * kg[r][i]; y4 += DP_B4[r] * kg[r][i]; }
        double yn = y0g[i] + h * y5;
        emax = fmax(emax, fabs(h * (y5 - y4)));
        ymax = fmax(ymax, fmax(fabs(y0g[i]), fabs(yn)));
        st->f.gam[i] = yn;
    }
    for (size_t i = 0; i < M; ++i) {
        double y5 = 0.0, y4 = 0.0;
        for (int r = 0; r < 7; ++r) { y5 += DP_B5[r] * kG[r][i]; y4 += DP_B4[r] * kG[r][i]; }
        double yn = y0G[i] + h * y5;
        emax = fmax(emax, fabs(h * (y5 - y4)));
        ymax = fmax(ymax, fmax(fabs(y0G[i]), fabs(yn)));
        G[i] = yn;
    }
    double err = emax / (atol + rtol * ymax);
    for (int i = 0; i < 7; ++i) { free(kg[i]); free(kG[i]); }
    free(y0g); free(y0G);
    return err;
}

/* chi^{mu nu}_{b k}, all 16 components (complex, interleaved): out[((off_b + k) * 16 + o) * 2].
 * Same quadrature as or_chi (C9); the bubble term carries tr(sigma^mu sigma^nu) / 2 =
 * delta_{mu nu} and is local (C8). */
void or_tri_chi(const OrStateT* st, double lam, double* outd) {
    const OrLattice* la = st->f.la;
    const int N = st->f.N;
    cx* out = (cx*)outd;
    double* y = (double*)malloc(sizeof(double) * (N + 1));
    double* Wn = (double*)calloc(N + 1, sizeof(double));
    int K = 0;
    y[K++] = lam;
    for (int i = 0; i < N; ++i) if (st->f.w[i] > lam) y[K++] = st->f.w[i];
    for (int k = 0; k + 1 < K; ++k) {
        double ya = y[k] + interp_odd(st->f.w, N, st->f.gam, y[k]);
        double yb = y[k + 1] + interp_odd(st->f.w, N, st->f.gam, y[k + 1]);
        double seg = (y[k + 1] - y[k]) / (ya * yb);
        Wn[k] += 0.5 * seg; Wn[k + 1] += 0.5 * seg;
    }
    Wn[K - 1] += 1.0 / (y[K - 1] + interp_odd(st->f.w, N, st->f.gam, y[K - 1]));
    double bubble = 0.0;
    for (int k = 0; k < K; ++k) bubble += Wn[k];
    bubble /= (2.0 * OR_PI);
    int M = 2 * K;
    double* xs = (double*)malloc(sizeof(double) * M);
    double* ws = (double*)malloc(sizeof(double) * M);
    for (int k = 0; k < K; ++k) { xs[k] = y[k]; ws[k] = Wn[k]; xs[K + k] = -y[k]; ws[K + k] = Wn[k]; }
    size_t base = 0;
    for (int b = 0; b < la->nb; ++b) {
        int ns = la->nsite[b];
        #pragma omp parallel for schedule(dynamic, 1)
        for (int k = 0; k < ns; ++k) {
            Site j = la->sites[b][k];
            int onsite = (j.b == b && j.n[0] == 0 && j.n[1] == 0 && j.n[2] == 0);
            int z[3] = {0, 0, 0};
            cx acc[16];
            for (int o = 0; o < 16; ++o) acc[o].re = acc[o].im = 0.0;
            for (int p = 0; p < M; ++p) for (int q = 0; q < M; ++q) {
                cx v[16], e[16];
                lookupT(st, b, j.n, j.b, xs[p] + xs[q], 0.0, xs[p] - xs[q], v);
                if (onsite) lookupT(st, b, z, b, xs[p] + xs[q], xs[q] - xs[p], 0.0, e);
                for (int o = 0; o < 16; ++o) {
                    cx F = {0.0, 0.0};
                    for (int x = 0; x < 16; ++x) {
                        F = cadd(F, cmul(g_tchi_dir[o][x], v[x]));
                        if (onsite) F = cadd(F, cscale(cmul(g_tchi_exc[o][x], e[x]), -1.0));
                    }
                    acc[o] = cadd(acc[o], cscale(F, ws[p] * ws[q]));
                }
            }
            for (int o = 0; o < 16; ++o) {
                cx r = cscale(acc[o], -1.0 / (16.0 * OR_PI * OR_PI));
                if (onsite && o / 4 == o % 4) r.re += bubble;
                out[(base + k) * 16 + o] = r;
            }
        }
        base += ns;
    }
    free(y); free(Wn); free(xs); free(ws);
}
