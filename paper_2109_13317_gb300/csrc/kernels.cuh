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
constexpr int kSeg = 8;            // lattice-sum table entries per work segment

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
    const int4* rpa;         // P: (rA, rB, permA, permB)
    const int* seg_start;    // nseg + 1: entry range of each segment
    const int* seg_r;        // nseg: output site of each segment
    const int* r_seg;        // Ns + 1: segment range of each output site
    int nseg;
};

__device__ __forceinline__ int perm_of(int packed, int c) { return (packed >> (2 * c)) & 3; }

__device__ __forceinline__ int pair_index(int si, int ui) { return si * (si + 1) / 2 + ui; }

// Nearest lesser / greater mesh points of x >= 0 and the interpolation weights of the
// paper's linear interpolation formula; constant extrapolation outside the mesh.
__device__ __forceinline__ void bracket(const double* __restrict__ w, int N, double x, int& lo, double& wlo, double& whi) {
    if (x <= w[0]) { lo = 0; wlo = 1.0; whi = 0.0; return; }
    if (x >= w[N - 1]) { lo = N - 2; wlo = 0.0; whi = 1.0; return; }
    int a = 0, b = N - 1;
    while (b - a > 1) {
        int m = (a + b) >> 1;
        if (w[m] <= x) a = m; else b = m;
    }
    lo = a;
    double h = w[a + 1] - w[a];
    wlo = (w[a + 1] - x) / h;
    whi = (x - w[a]) / h;
}

// gamma(x), odd, linear interpolation on |x| with constant extrapolation, gamma(0) = 0.
__device__ __forceinline__ double interp_odd(const double* __restrict__ w, int N, const double* __restrict__ f, double x) {
    if (x == 0.0) return 0.0;
    double ax = fabs(x);
    int lo; double wl, wh;
    bracket(w, N, ax, lo, wl, wh);
    double v = wl * f[lo] + wh * f[lo + 1];
    return x < 0.0 ? -v : v;
}

// Lookup descriptor of Gamma(s, t, u) for one frequency triple: the symmetry relations of
// Eq. (frg:parametrizationBasis2p) bring the arguments to s, t, u >= 0, s >= u (t -> -t is
// a no-op on spin-diagonal functions; s -> -s and u -> -u exchange the two sites), then the
// eight trilinear corners with their offsets into the state (site 0, component 0) and
// weights; corners below the s = u diagonal read through the s <-> u relation, which flips
// the sign of the density component.
template <typename T>
struct Desc {
    int off[8];
    T wd[8];   // weight applied to the density component
    T ws[8];   // weight applied to the spin components
    int swap;
};

template <typename T>
__device__ __forceinline__ void make_desc(double s, double t, double u, const double* __restrict__ w, const Geo& g,
                                          Desc<T>& d) {
    int swap = 0;
    if (t < 0.0) t = -t;
    if (s < 0.0) { s = -s; swap ^= 1; }
    if (u < 0.0) { u = -u; swap ^= 1; }
    double flip = 1.0;
    if (s < u) { double tmp = s; s = u; u = tmp; flip = -1.0; }
    int sl, tl, ul;
    double sw[2], tw[2], uw[2];
    bracket(w, g.N, s, sl, sw[0], sw[1]);
    bracket(w, g.N, t, tl, tw[0], tw[1]);
    bracket(w, g.N, u, ul, uw[0], uw[1]);
    const int row = g.nc * g.Ns;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        int a = k & 1, b = (k >> 1) & 1, c = (k >> 2) & 1;
        int si = sl + a, ti = tl + b, ui = ul + c;
        double wt = sw[a] * tw[b] * uw[c];
        double sg = flip;
        int p;
        if (si >= ui) p = pair_index(si, ui);
        else { p = pair_index(ui, si); sg = -flip; }
        d.off[k] = (p * g.N + ti) * row;
        d.wd[k] = (T)(wt * sg);
        d.ws[k] = (T)wt;
    }
    d.swap = swap;
}

// Value of component c of the pair (ref, rep_r) at the descriptor's frequencies.
template <typename T>
__device__ __forceinline__ T row_value(const T* __restrict__ G, const Desc<T>& d, const Tabs& tb, const Geo& g, int r, int c) {
    int rs = r, cs = c;
    if (d.swap) { rs = tb.swap_r[r]; cs = perm_of(tb.swap_perm[r], c); }
    const T* base = G + cs * g.Ns + rs;
    T acc = 0;
    if (c == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) acc += d.wd[k] * base[d.off[k]];
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) acc += d.ws[k] * base[d.off[k]];
    }
    return acc;
}

}  // namespace dev
}  // namespace sr
