// Device kernels of the pf-FRG flow right-hand side (internal header, sm_103a).
//
// Equations: arXiv:2109.13317, Sec. 3 (flow of Sigma and of Gamma^{mu nu}_{i1 i2}(s,t,u)),
// Sec. 4.2 (linear / trilinear frequency interpolation with constant extrapolation,
// trapezoidal integration on the mesh nodes), Sec. 4.3 (Euler).  Sigma = -i gamma with
// gamma real and odd; all SU2 / XYZ arithmetic is real.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sr {
namespace dev {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxFreq = 256;      // largest supported mesh

// Flow-wide constants passed by value to every kernel.
struct Geo {
    int N;        // positive frequencies
    int Ns;       // irreducible sites
    int nc;       // stored spin components (2 SU2, 4 XYZ)
    int npair;    // N (N + 1) / 2
    int nmax;     // node capacity per (channel, transfer frequency): 2N + 8
    long nent;    // Gamma entries
};

// Tables of the lattice (device pointers).
struct Tabs {
    const int* swap_r;       // Ns: irreducible site of the exchanged pair
    const int* swap_perm;    // Ns: packed component map of the exchanged pair
    const int* onsite_perm;  // Ns: packed component map of (rep, rep) onto site 0
    const int* mult;         // Ns: Hartree multiplicity
    const int2* prod;        // nprod: distinct lattice-sum products (row index A, row index B)
    const int* gath_off;     // Ns * nc + 1: product range of each output (site, component)
    const int* gath_idx;     // P * nc: product of each table entry, grouped by output
    int nprod;
    const double* invh;      // N - 1: 1 / (w[a+1] - w[a])
};

__device__ __forceinline__ int perm_of(int packed, int c) { return (packed >> (2 * c)) & 3; }

__device__ __forceinline__ int pair_index(int si, int ui) { return si * (si + 1) / 2 + ui; }

// Nearest lesser / greater mesh points of x >= 0 and the interpolation weights of the
// paper's linear interpolation formula (with the reciprocal interval width); constant
// extrapolation outside the mesh.  At a mesh point one weight is exactly zero.
__device__ __forceinline__ void bracket(const double* __restrict__ w, const double* __restrict__ invh, int N, double x,
                                        int& lo, double& wlo, double& whi) {
    if (x <= w[0]) { lo = 0; wlo = 1.0; whi = 0.0; return; }
    if (x >= w[N - 1]) { lo = N - 2; wlo = 0.0; whi = 1.0; return; }
    int a = 0, b = N - 1;
    while (b - a > 1) {
        int m = (a + b) >> 1;
        if (w[m] <= x) a = m; else b = m;
    }
    lo = a;
    wlo = (w[a + 1] - x) * invh[a];
    whi = (x - w[a]) * invh[a];
}

// gamma(x), odd, linear interpolation on |x| with constant extrapolation, gamma(0) = 0.
__device__ __forceinline__ double interp_odd(const double* __restrict__ w, const double* __restrict__ invh, int N,
                                             const double* __restrict__ f, double x) {
    if (x == 0.0) return 0.0;
    double ax = fabs(x);
    int lo; double wl, wh;
    bracket(w, invh, N, ax, lo, wl, wh);
    double v = wl * f[lo] + wh * f[lo + 1];
    return x < 0.0 ? -v : v;
}

// Lookup descriptor of Gamma(s, t, u) for one frequency triple: the symmetry relations of
// Eq. (frg:parametrizationBasis2p) bring the arguments to s, t, u >= 0, s >= u (t -> -t is
// a no-op on spin-diagonal functions; s -> -s and u -> -u exchange the two sites), then the
// trilinear corners with non-zero weight (one argument of every row of the flow equations
// is a mesh frequency, so four corners remain), their offsets into the state (site 0,
// component 0) and weights; corners below the s = u diagonal read through the s <-> u
// relation, which flips the sign of the density component.
template <typename T>
struct Desc {
    int n;      // corners with non-zero weight
    int swap;
    int off[8];
    T wd[8];    // weight applied to the density component
    T ws[8];    // weight applied to the spin components
};

template <typename T>
__device__ __forceinline__ void make_desc(double s, double t, double u, const double* __restrict__ w,
                                          const double* __restrict__ invh, const Geo& g, Desc<T>& d) {
    int swap = 0;
    if (t < 0.0) t = -t;
    if (s < 0.0) { s = -s; swap ^= 1; }
    if (u < 0.0) { u = -u; swap ^= 1; }
    double flip = 1.0;
    if (s < u) { double tmp = s; s = u; u = tmp; flip = -1.0; }
    int ix[3][2], nx[3];
    double wx[3][2];
    const double arg[3] = {s, t, u};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int lo; double w0, w1;
        bracket(w, invh, g.N, arg[a], lo, w0, w1);
        if (w1 == 0.0) { nx[a] = 1; ix[a][0] = lo; wx[a][0] = w0; }
        else if (w0 == 0.0) { nx[a] = 1; ix[a][0] = lo + 1; wx[a][0] = w1; }
        else { nx[a] = 2; ix[a][0] = lo; wx[a][0] = w0; ix[a][1] = lo + 1; wx[a][1] = w1; }
    }
    const int row = g.nc * g.Ns;
    int k = 0;
    for (int a = 0; a < nx[0]; ++a)
        for (int b = 0; b < nx[1]; ++b)
            for (int c = 0; c < nx[2]; ++c) {
                int si = ix[0][a], ti = ix[1][b], ui = ix[2][c];
                double wt = wx[0][a] * wx[1][b] * wx[2][c];
                double sg = flip;
                int p;
                if (si >= ui) p = pair_index(si, ui);
                else { p = pair_index(ui, si); sg = -flip; }
                d.off[k] = (p * g.N + ti) * row;
                d.wd[k] = (T)(wt * sg);
                d.ws[k] = (T)wt;
                ++k;
            }
    d.n = k;
    d.swap = swap;
}

// Value of component c of the pair (ref, rep_r) at the descriptor's frequencies.
template <typename T>
__device__ __forceinline__ T row_value(const T* __restrict__ G, const Desc<T>& d, const Tabs& tb, const Geo& g, int r, int c) {
    int rs = r, cs = c;
    if (d.swap) { rs = tb.swap_r[r]; cs = perm_of(tb.swap_perm[r], c); }
    const T* base = G + cs * g.Ns + rs;
    const T* wgt = c == 0 ? d.wd : d.ws;
    T acc = 0;
    for (int k = 0; k < d.n; ++k) acc += wgt[k] * base[d.off[k]];
    return acc;
}

}  // namespace dev
}  // namespace sr
