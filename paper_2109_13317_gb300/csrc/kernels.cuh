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
    int nsp;          // sites padded to a multiple of 4 (FP32 shadow layout)
    long nentp;       // entries of the padded FP32 shadow
    float log2w0;     // log2(w[0])
    float inv_dlog2;  // (N - 1) / log2(w[N-1] / w[0]): interval guess for a log-spaced mesh
    unsigned div4;    // ceil(2^32 / (nsp / 4)) (0 when nsp = 4): n / (nsp / 4) = __umulhi(n, div4)
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
    const double* w;         // N: mesh
    const float* wf;         // N: mesh (FP32)
    const float* invhf;      // N - 1: 1 / (w[a+1] - w[a]) (FP32)
    const int2* prodp;       // nprod: lattice-sum products in the padded layout (c * nsp + r)
    const int* dgath_idx;    // P * nc: dense-contraction index c * nsp^2 + rA * nsp + rB (SU2)
};

// Forward-mode dual number: a value and its derivatives along P parameter directions.  The
// flow kernels are written once for a scalar type T; with T = Dual<P> every arithmetic step
// also propagates the tangents (the tangent-linear flow), while every decision (interval,
// sign, support) is taken on frequencies, which carry no tangent.
template <int P>
struct Dual {
    double v;
    double d[P];
    Dual() = default;
    __host__ __device__ Dual(double x) : v(x) {
        for (int i = 0; i < P; ++i) d[i] = 0.0;
    }
};
template <int P> __host__ __device__ inline Dual<P> operator+(const Dual<P>& a, const Dual<P>& b) {
    Dual<P> r; r.v = a.v + b.v; for (int i = 0; i < P; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int P> __host__ __device__ inline Dual<P> operator-(const Dual<P>& a, const Dual<P>& b) {
    Dual<P> r; r.v = a.v - b.v; for (int i = 0; i < P; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int P> __host__ __device__ inline Dual<P> operator-(const Dual<P>& a) {
    Dual<P> r; r.v = -a.v; for (int i = 0; i < P; ++i) r.d[i] = -a.d[i]; return r; }
template <int P> __host__ __device__ inline Dual<P> operator*(const Dual<P>& a, const Dual<P>& b) {
    Dual<P> r; r.v = a.v * b.v; for (int i = 0; i < P; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int P> __host__ __device__ inline Dual<P> operator*(double a, const Dual<P>& b) {
    Dual<P> r; r.v = a * b.v; for (int i = 0; i < P; ++i) r.d[i] = a * b.d[i]; return r; }
template <int P> __host__ __device__ inline Dual<P> operator*(const Dual<P>& b, double a) { return a * b; }
template <int P> __host__ __device__ inline Dual<P> operator/(const Dual<P>& a, const Dual<P>& b) {
    Dual<P> r; r.v = a.v / b.v; const double ib = 1.0 / b.v;
    for (int i = 0; i < P; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib; return r; }
template <int P> __host__ __device__ inline Dual<P> operator/(double a, const Dual<P>& b) { return Dual<P>(a) / b; }
template <int P> __host__ __device__ inline Dual<P> operator/(const Dual<P>& a, double b) {
    Dual<P> r; r.v = a.v / b; for (int i = 0; i < P; ++i) r.d[i] = a.d[i] / b; return r; }
template <int P> __host__ __device__ inline Dual<P> operator+(double a, const Dual<P>& b) { return Dual<P>(a) + b; }
template <int P> __host__ __device__ inline Dual<P> operator+(const Dual<P>& b, double a) { return b + Dual<P>(a); }
template <int P> __host__ __device__ inline Dual<P> operator-(double a, const Dual<P>& b) { return Dual<P>(a) - b; }
template <int P> __host__ __device__ inline Dual<P> operator-(const Dual<P>& b, double a) { return b - Dual<P>(a); }
template <int P> __host__ __device__ inline Dual<P>& operator+=(Dual<P>& a, const Dual<P>& b) { a = a + b; return a; }
template <int P> __host__ __device__ inline Dual<P>& operator-=(Dual<P>& a, const Dual<P>& b) { a = a - b; return a; }
template <int P> __host__ __device__ inline Dual<P>& operator*=(Dual<P>& a, const Dual<P>& b) { a = a * b; return a; }

__host__ __device__ inline double value_of(double x) { return x; }
__host__ __device__ inline float value_of(float x) { return x; }
template <int P> __host__ __device__ inline double value_of(const Dual<P>& x) { return x.v; }

// Type of interpolation weights for a state scalar T (weights carry no tangent).
template <typename T> struct WeightOf { using type = T; };
template <int P> struct WeightOf<Dual<P>> { using type = double; };

constexpr int kTan = 2;   // tangent directions of the tangent-linear flow
using DualT = Dual<kTan>;

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
template <typename T>
__device__ __forceinline__ T interp_odd(const double* __restrict__ w, const double* __restrict__ invh, int N,
                                        const T* __restrict__ f, double x) {
    if (x == 0.0) return T(0.0);
    double ax = fabs(x);
    int lo; double wl, wh;
    bracket(w, invh, N, ax, lo, wl, wh);
    T v = wl * f[lo] + wh * f[lo + 1];
    return x < 0.0 ? T(-v) : v;
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

// Interval guess for x inside the mesh, from the log spacing (exact for a logarithmic mesh
// up to one step; any mesh is then corrected by the exact comparisons of the caller).
__device__ __forceinline__ int interval_guess(const Geo& g, float x) {
    int k = __float2int_rd((__log2f(x) - g.log2w0) * g.inv_dlog2);
    return max(0, min(k, g.N - 2));
}

// Corners and weights of one axis: the interval [w_k, w_k+1] with w_k <= x < w_k+1 and the
// paper's linear weights; one corner at a mesh point or outside the mesh (constant
// extrapolation).  FP64 for T = double (decisions identical to a binary search), FP32
// arithmetic for T = float.
template <typename T>
__device__ __forceinline__ void axis_weights(const Tabs& tb, const Geo& g, double x, int& n, int* ix, T* wx) {
    const int N = g.N;
    if constexpr (sizeof(T) == 8) {
        const double* w = tb.w;
        // x >= 0 (make_desc folds the signs) and the mesh is positive, so the comparisons run
        // on the bit patterns, which order like the values (a -0 orders below every mesh
        // point, as 0 does), on the integer pipe instead of the FP64 pipe
        const long long xb = __double_as_longlong(x);
        auto below = [&](int i) { return xb < __double_as_longlong(w[i]); };   // x < w[i]
        if (below(0) || xb == __double_as_longlong(w[0])) { n = 1; ix[0] = 0; wx[0] = (T)1; return; }   // x <= w[0]
        if (!below(N - 1)) { n = 1; ix[0] = N - 1; wx[0] = (T)1; return; }                            // x >= w[N-1]
        int k = interval_guess(g, (float)x);
        while (k > 0 && below(k)) --k;
        while (k < N - 2 && !below(k + 1)) ++k;
        const double w1 = (x - w[k]) * tb.invh[k];
        if ((__double_as_longlong(w1) & 0x7fffffffffffffffLL) == 0) { n = 1; ix[0] = k; wx[0] = (T)1; return; }   // w1 == 0
        n = 2; ix[0] = k; ix[1] = k + 1;
        wx[0] = (T)((w[k + 1] - x) * tb.invh[k]);
        wx[1] = (T)w1;
    } else {
        const float* w = tb.wf;
        const float xf = (float)x;
        if (xf <= w[0]) { n = 1; ix[0] = 0; wx[0] = (T)1; return; }
        if (xf >= w[N - 1]) { n = 1; ix[0] = N - 1; wx[0] = (T)1; return; }
        int k = interval_guess(g, xf);
        while (k > 0 && xf < w[k]) --k;
        while (k < N - 2 && xf >= w[k + 1]) ++k;
        const float w1 = (xf - w[k]) * tb.invhf[k];
        if (w1 == 0.0f) { n = 1; ix[0] = k; wx[0] = (T)1; return; }
        n = 2; ix[0] = k; ix[1] = k + 1;
        wx[0] = (T)((w[k + 1] - xf) * tb.invhf[k]);
        wx[1] = (T)w1;
    }
}

// FP32 version of axis_weights for an FP32 argument (the mixed-precision vertex kernel).
__device__ __forceinline__ void axis_weights_f(const Tabs& tb, const Geo& g, float xf, int& n, int* ix, float* wx) {
    const int N = g.N;
    const float* w = tb.wf;
    if (xf <= w[0]) { n = 1; ix[0] = 0; wx[0] = 1.0f; return; }
    if (xf >= w[N - 1]) { n = 1; ix[0] = N - 1; wx[0] = 1.0f; return; }
    int k = interval_guess(g, xf);
    while (k > 0 && xf < w[k]) --k;
    while (k < N - 2 && xf >= w[k + 1]) ++k;
    const float w1 = (xf - w[k]) * tb.invhf[k];
    if (w1 == 0.0f) { n = 1; ix[0] = k; wx[0] = 1.0f; return; }
    n = 2; ix[0] = k; ix[1] = k + 1;
    wx[0] = (w[k + 1] - xf) * tb.invhf[k];
    wx[1] = w1;
}

// Corners of a descriptor whose exact axis EA (0 s, 1 t, 2 u) is known at compile time, so
// that every per-axis index is static (the descriptor arithmetic stays in registers).
// Corners are enumerated with the s axis outermost and the u axis innermost.
template <int EA, bool SCALE, typename T>
__device__ __forceinline__ void desc_corners(double s, double t, double u, int ex_idx, bool flip, const Tabs& tb,
                                             const Geo& g, Desc<T>& d, T scale) {
    constexpr int A0 = EA == 0 ? 1 : 0, A1 = EA == 2 ? 1 : 2;
    const double x0 = A0 == 0 ? s : t, x1 = A1 == 1 ? t : u;
    int i0[2], i1[2], n0, n1;
    T v0[2], v1[2];
    axis_weights<T>(tb, g, x0, n0, i0, v0);
    axis_weights<T>(tb, g, x1, n1, i1, v1);
    if constexpr (SCALE) {   // a factor of every corner weight (a node weight), on one axis
        v0[0] *= scale;
        if (n0 > 1) v0[1] *= scale;
    }
    const int row = g.nc * g.Ns;
    int k = 0;
#pragma unroll
    for (int b0 = 0; b0 < 2; ++b0) {
        if (b0 >= n0) break;
#pragma unroll
        for (int b1 = 0; b1 < 2; ++b1) {
            if (b1 >= n1) break;
            const int js = EA == 0 ? ex_idx : i0[b0];
            const int jt = EA == 1 ? ex_idx : (A0 == 1 ? i0[b0] : i1[b1]);
            const int ju = EA == 2 ? ex_idx : i1[b1];
            const T wt = v0[b0] * v1[b1];
            bool neg = flip;
            int p;
            if (js >= ju) p = pair_index(js, ju);
            else { p = pair_index(ju, js); neg = !neg; }
            d.off[k] = (p * g.N + jt) * row;
            d.wd[k] = neg ? -wt : wt;
            d.ws[k] = wt;
            ++k;
        }
    }
    d.n = k;
}

// Descriptor of Gamma(s, t, u).  ex_slot (0 s, 1 t, 2 u) names an argument known to be the
// mesh frequency w[ex_idx] (or 0, clamped to w[0]), which needs no interval search.  SCALE:
// every corner weight carries the factor `scale` (the node weight of an integration row).
template <typename T, bool SCALE = false>
__device__ __forceinline__ void make_desc(double s, double t, double u, int ex_slot, int ex_idx, const Tabs& tb,
                                          const Geo& g, Desc<T>& d, T scale = T(1)) {
    // sign tests and the s < u comparison on the bit patterns (integer pipe): x < 0 is a set
    // sign bit on a value other than -0; after the folding both are >= 0 (or -0, compared as 0
    // with the sign bit masked), where the bit patterns order like the values
    constexpr long long kMag = 0x7fffffffffffffffLL;
    auto negative = [](double x) { const long long b = __double_as_longlong(x); return b < 0 && (b & kMag) != 0; };
    int swap = 0;
    if (negative(t)) t = -t;
    if (negative(s)) { s = -s; swap ^= 1; }
    if (negative(u)) { u = -u; swap ^= 1; }
    bool flip = false;
    if ((__double_as_longlong(s) & kMag) < (__double_as_longlong(u) & kMag)) {
        double tmp = s; s = u; u = tmp; flip = true; if (ex_slot != 1) ex_slot = 2 - ex_slot;
    }
    if (ex_slot == 0) desc_corners<0, SCALE, T>(s, t, u, ex_idx, flip, tb, g, d, scale);
    else if (ex_slot == 1) desc_corners<1, SCALE, T>(s, t, u, ex_idx, flip, tb, g, d, scale);
    else desc_corners<2, SCALE, T>(s, t, u, ex_idx, flip, tb, g, d, scale);
    d.swap = swap;
}

// Four-corner descriptor of the FP32 kernel (every row there has one argument on the mesh,
// so at most four corners carry weight; unused corners have weight zero and offset zero).
struct __align__(16) DescF {
    int off[4];
    float wd[4];
    float ws[4];
    int swap;
    int pad[3];
};

// Corners of the FP32 descriptor with the exact axis EA known at compile time, so that every
// per-axis array index is static and the descriptor stays in registers.
template <int EA>
__device__ __forceinline__ void desc4_corners(float s, float t, float u, int ex_idx, bool flip, const Tabs& tb,
                                              const Geo& g, int rowp, DescF& d) {
    constexpr int A0 = EA == 0 ? 1 : 0, A1 = EA == 2 ? 1 : 2;
    const float x0 = A0 == 0 ? s : t, x1 = A1 == 1 ? t : u;
    int i0[2], i1[2], n0, n1;
    float v0[2], v1[2];
    axis_weights_f(tb, g, x0, n0, i0, v0);
    if (n0 == 1) { i0[1] = i0[0]; v0[1] = 0.0f; }
    axis_weights_f(tb, g, x1, n1, i1, v1);
    if (n1 == 1) { i1[1] = i1[0]; v1[1] = 0.0f; }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int b0 = k & 1, b1 = k >> 1;
        const int js = EA == 0 ? ex_idx : i0[b0];
        const int jt = EA == 1 ? ex_idx : (A0 == 1 ? i0[b0] : i1[b1]);
        const int ju = EA == 2 ? ex_idx : i1[b1];
        const float wt = v0[b0] * v1[b1];
        bool neg = flip;
        int p;
        if (js >= ju) p = pair_index(js, ju);
        else { p = pair_index(ju, js); neg = !neg; }
        d.off[k] = wt != 0.0f ? (p * g.N + jt) * rowp : 0;
        d.wd[k] = neg ? -wt : wt;
        d.ws[k] = wt;
    }
}

// FP32 descriptor of Gamma(s, t, u) with one exact argument (ex_slot 0 s, 1 t, 2 u, the mesh
// frequency w[ex_idx]): symmetry folding as in make_desc, then four corners over the other two
// axes (zero-weight corners kept, pointing at offset 0).
__device__ __forceinline__ void make_desc4(float s, float t, float u, int ex_slot, int ex_idx, const Tabs& tb,
                                           const Geo& g, int rowp, DescF& d) {
    int swap = 0;
    if (t < 0.0f) t = -t;
    if (s < 0.0f) { s = -s; swap ^= 1; }
    if (u < 0.0f) { u = -u; swap ^= 1; }
    bool flip = false;
    if (s < u) { float tmp = s; s = u; u = tmp; flip = true; if (ex_slot != 1) ex_slot = 2 - ex_slot; }
    if (ex_slot == 0) desc4_corners<0>(s, t, u, ex_idx, flip, tb, g, rowp, d);
    else if (ex_slot == 1) desc4_corners<1>(s, t, u, ex_idx, flip, tb, g, rowp, d);
    else desc4_corners<2>(s, t, u, ex_idx, flip, tb, g, rowp, d);
    d.swap = swap;
}

// Store a descriptor built in registers to shared memory as four 16-byte chunks, chunk order
// rotated by (lane >> 1) & 3 so that the eight lanes of a quarter warp, whose descriptors lie
// 64 bytes apart, write eight distinct bank quads.
__device__ __forceinline__ void store_desc4(DescF* dst, const DescF& d, int lane) {
    const int4 c0 = *reinterpret_cast<const int4*>(d.off);
    const int4 c1 = *reinterpret_cast<const int4*>(d.wd);
    const int4 c2 = *reinterpret_cast<const int4*>(d.ws);
    const int4 c3 = make_int4(d.swap, 0, 0, 0);
    int4* out = reinterpret_cast<int4*>(dst);
    const int rot = (lane >> 1) & 3;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int k = (j + rot) & 3;
        const int4 v = k == 0 ? c0 : (k == 1 ? c1 : (k == 2 ? c2 : c3));
        out[k] = v;
    }
}

// Value of component c of the pair (ref, rep_r) at the descriptor's frequencies.
template <typename T, typename W>
__device__ __forceinline__ T row_value(const T* __restrict__ G, const Desc<W>& d, const Tabs& tb, const Geo& g, int r, int c) {
    int rs = r, cs = c;
    if (d.swap) { rs = tb.swap_r[r]; cs = perm_of(tb.swap_perm[r], c); }
    const T* base = G + cs * g.Ns + rs;
    const W* wgt = c == 0 ? d.wd : d.ws;
    T acc = T(0.0);
    for (int k = 0; k < d.n; ++k) acc += wgt[k] * base[d.off[k]];
    return acc;
}

}  // namespace dev
}  // namespace sr
