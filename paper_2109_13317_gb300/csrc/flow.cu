// pf-FRG flow on one GB300 GPU: kernels of the right-hand side, Euler / Dormand-Prince
// stepping, the correlation measurement, and the C ABI declared in include/sr.h.
//
// Right-hand side, per cutoff Lambda (arXiv:2109.13317, Sec. 3 and 4):
//   1. k_sigma_rhs     dgamma(w_n): Hartree lattice sum + Fock on-site term at the two
//                      delta points w2 = +-Lambda of the single-scale propagator.
//   2. k_channel_nodes per channel (s, t, u) and transfer frequency: the w' integration
//                      nodes and weights -- four exact delta points of S and the trapezoid
//                      rule on the regular Katanin part -- shared by every vertex entry
//                      with that transfer frequency (the paper's buffered weights).
//   3. k_gamma_rhs     one CTA per stored (s, u, t) triple: all sites and components.
//                      Per block of integration nodes it builds the interpolated vertex
//                      rows over all irreducible sites in shared memory, then the s / u
//                      channel products, the t-channel on-site terms, and the lattice sum
//                      sum_j Gamma_{i1 j} Gamma_{j i2} through the tabulated site list.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "tc.cuh"
#include "lattice.hpp"
#include "sr.h"

using namespace sr::dev;
namespace tc = sr::tc;

// ----------------------------------------------------------------------------- errors

static thread_local std::string g_err;

static sr_status fail(sr_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(SR_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" const char* sr_last_error(void) { return g_err.c_str(); }

// ----------------------------------------------------------------------------- kernels

namespace {

constexpr int kQC = 16;       // integration nodes per shared-memory block
constexpr int kThreads = 128;

// Propagator products with Sigma = -i gamma: g(a) g(b) and g(a) r(b), r = -g^2 dSigma/dLambda.
template <typename T>
__device__ __forceinline__ T prop_gg(const double* w, const double* invh, int N, const T* gam, double a, double b) {
    const T ga = a + interp_odd(w, invh, N, gam, a);
    const T gb = b + interp_odd(w, invh, N, gam, b);
    return -1.0 / (ga * gb);
}
template <typename T>
__device__ __forceinline__ T prop_gr(const double* w, const double* invh, int N, const T* gam, const T* dgam, double a, double b) {
    const T ga = a + interp_odd(w, invh, N, gam, a);
    const T gb = b + interp_odd(w, invh, N, gam, b);
    const T db = interp_odd(w, invh, N, dgam, b);
    return -db / (ga * gb * gb);
}

__device__ __forceinline__ bool in_support(double lam, int ch, double v, double m) {
    if (fabs(m) < lam) return false;
    if (ch == 0) return fabs(v - m) >= lam;
    if (ch == 1) return fabs(m - v) >= lam;
    return fabs(v + m) >= lam;
}

template <typename T>
__device__ __forceinline__ T preg(const double* w, const double* invh, int N, const T* gam, const T* dgam, int ch, double v, double x) {
    if (ch == 0) return prop_gr(w, invh, N, gam, dgam, x, v - x) + prop_gr(w, invh, N, gam, dgam, v - x, x);
    if (ch == 1) return prop_gr(w, invh, N, gam, dgam, x, x - v) + prop_gr(w, invh, N, gam, dgam, x - v, x);
    return prop_gr(w, invh, N, gam, dgam, x, v + x) + prop_gr(w, invh, N, gam, dgam, v + x, x);
}

// Integration nodes of one channel (ch = 0 s, 1 t, 2 u) at transfer frequency w[vi]; one
// block per (channel, frequency).  The regular-part points ({+-w_n} merged with the clipped
// break points) are placed by rank, their trapezoid weights and propagator values computed
// in parallel, then compacted in order.
template <typename T>
__device__ void channel_nodes_block(Geo g, const double* __restrict__ w, const double* __restrict__ invh,
                                    const T* __restrict__ gam, const T* __restrict__ dgam, double lam,
                                    double* __restrict__ nx, T* __restrict__ nW, float* __restrict__ nWf,
                                    int* __restrict__ ncount, const int id, float* __restrict__ nxf = nullptr,
                                    double* __restrict__ ntw = nullptr) {
    __shared__ double pts[2 * kMaxFreq + 4];
    __shared__ double twt[2 * kMaxFreq + 4];
    __shared__ __align__(16) unsigned char val_raw[sizeof(T) * (2 * kMaxFreq + 4)];
    T* val = reinterpret_cast<T*>(val_raw);
    __shared__ unsigned char keep[2 * kMaxFreq + 4];
    __shared__ double bp[4];
    const int ch = id / g.N, vi = id % g.N, N = g.N;
    const double v = w[vi];
    double* X = nx + (size_t)id * g.nmax;
    T* Wt = nW + (size_t)id * g.nmax;
    float* Wf = nWf ? nWf + (size_t)id * g.nmax : nullptr;
    const double inv2pi = 1.0 / (2.0 * kPi);
    const double wmax = w[N - 1];
    const int m = 2 * N + 4;
    if (threadIdx.x == 0) {
        // delta points of the single-scale propagator, theta(0) = 1; a point whose partner
        // propagator lies below the cutoff (theta = 0) contributes exactly zero
        int n = 0;
        for (int sg = 0; sg < 2; ++sg) {
            double L = sg == 0 ? lam : -lam;
            double a;
            if (ch == 0) {          // G(w) S(s - w): w = s - L;  G(s - w) S(w): w = L
                a = v - L;
                const T vv = (fabs(a) - lam >= 0.0) ? T(prop_gg(w, invh, N, gam, a, L) * inv2pi) : T(0.0);
                X[n] = a; Wt[n] = vv; ++n;
                X[n] = L; Wt[n] = vv; ++n;
            } else if (ch == 1) {   // G(w) S(w - t): w = t + L;  G(w - t) S(w): w = L
                a = v + L;
                X[n] = a; Wt[n] = (fabs(a) - lam >= 0.0) ? T(prop_gg(w, invh, N, gam, a, L) * inv2pi) : T(0.0); ++n;
                a = L - v;
                X[n] = L; Wt[n] = (fabs(a) - lam >= 0.0) ? T(prop_gg(w, invh, N, gam, a, L) * inv2pi) : T(0.0); ++n;
            } else {                // G(w) S(u + w): w = L - u;  G(u + w) S(w): w = L
                a = L - v;
                X[n] = a; Wt[n] = (fabs(a) - lam >= 0.0) ? T(prop_gg(w, invh, N, gam, a, L) * inv2pi) : T(0.0); ++n;
                a = v + L;
                X[n] = L; Wt[n] = (fabs(a) - lam >= 0.0) ? T(prop_gg(w, invh, N, gam, a, L) * inv2pi) : T(0.0); ++n;
            }
        }
        // break points, clipped to [-w_max, w_max], in ascending order (insertion order on ties)
        double q[4];
        if (ch == 2) { q[0] = lam; q[1] = -lam; q[2] = -v + lam; q[3] = -v - lam; }
        else { q[0] = lam; q[1] = -lam; q[2] = v + lam; q[3] = v - lam; }
        for (int i = 0; i < 4; ++i) {
            double c = q[i];
            if (c > wmax) c = wmax;
            if (c < -wmax) c = -wmax;
            int j = i;
            while (j > 0 && bp[j - 1] > c) { bp[j] = bp[j - 1]; --j; }
            bp[j] = c;
        }
    }
    __syncthreads();
    // place every point by rank: a mesh point precedes break points of equal value
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) {
        const double x = i < N ? -w[N - 1 - i] : w[i - N];
        int r = i;
        for (int j = 0; j < 4; ++j) r += bp[j] < x;
        pts[r] = x;
    }
    for (int j = threadIdx.x; j < 4; j += blockDim.x) {
        const double x = bp[j];
        int lo = 0, hi = 2 * N;   // count mesh points <= x
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const double y = mid < N ? -w[N - 1 - mid] : w[mid - N];
            if (y <= x) lo = mid + 1; else hi = mid;
        }
        pts[lo + j] = x;
    }
    __syncthreads();
    // trapezoid weight of each point over its supported neighbouring segments, times the
    // regular propagator pair without theta
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double wgt = 0.0;
        if (i > 0 && pts[i] > pts[i - 1] && in_support(lam, ch, v, 0.5 * (pts[i] + pts[i - 1])))
            wgt += 0.5 * (pts[i] - pts[i - 1]);
        if (i + 1 < m && pts[i + 1] > pts[i] && in_support(lam, ch, v, 0.5 * (pts[i] + pts[i + 1])))
            wgt += 0.5 * (pts[i + 1] - pts[i]);
        val[i] = wgt == 0.0 ? T(0.0) : T(wgt * preg(w, invh, N, gam, dgam, ch, v, pts[i]) * inv2pi);
        keep[i] = wgt != 0.0;
        twt[i] = wgt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int n = 4;
        for (int i = 0; i < m; ++i) {
            if (!keep[i]) continue;
            X[n] = pts[i];
            Wt[n] = val[i];
            if (ntw) ntw[(size_t)id * g.nmax + n] = twt[i];
            ++n;
        }
        if (Wf)
            for (int i = 0; i < n; ++i) Wf[i] = (float)value_of(Wt[i]);
        if (nxf)
            for (int i = 0; i < n; ++i) nxf[(size_t)id * g.nmax + i] = (float)X[i];
        ncount[id] = n;
    }
}

template <typename T>
__global__ void k_channel_nodes(Geo g, const double* __restrict__ w, const double* __restrict__ invh,
                                const T* __restrict__ gam, const T* __restrict__ dgam, double lam,
                                double* __restrict__ nx, T* __restrict__ nW, float* __restrict__ nWf,
                                int* __restrict__ ncount, float* __restrict__ nxf, double* __restrict__ ntw = nullptr) {
    channel_nodes_block<T>(g, w, invh, gam, dgam, lam, nx, nW, nWf, ncount, blockIdx.x, nxf, ntw);
}

// Deterministic block sum (fixed reduction tree for a fixed block size) of NV scalars of
// type T (doubles or dual numbers, reduced component by component); red holds
// NV * (sizeof(T) / 8) * 32 doubles.
template <typename T, int NV>
__device__ void block_sum(T (&v)[NV], double* red) {
    constexpr int K = NV * (int)(sizeof(T) / sizeof(double));
    double* a = reinterpret_cast<double*>(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < K; ++k) red[k * 32 + wid] = a[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < K; ++k) {
            double acc = 0.0;
            for (int i = 0; i < nw; ++i) acc += red[k * 32 + i];
            a[k] = acc;
        }
}

// Flow of the self-energy, one block per mesh frequency w_n:
// dgamma(w) = -(1/2pi) sum_{w2 = +-Lambda} H(w, w2) / (w2 + gamma(w2)),
// H = 2 sum_j Gamma^00_{ref j}(w+w2, 0, w-w2) - sum_c f_c Gamma^cc_{ref ref}(w+w2, w2-w, 0).
template <typename T>
__device__ void sigma_rhs_block(Geo g, Tabs tb, const double* __restrict__ w, const T* __restrict__ gam,
                                const T* __restrict__ G, double lam, T* __restrict__ dgam, const int n) {
    __shared__ double red[2 * 32 * (sizeof(T) / sizeof(double))];
    const double w1 = w[n];
    T H[2] = {T(0.0), T(0.0)};
    for (int sg = 0; sg < 2; ++sg) {
        const double w2 = sg == 0 ? lam : -lam;
        Desc<double> d;
        make_desc(w1 + w2, 0.0, w1 - w2, 1, 0, tb, g, d);
        T h = T(0.0);
        for (int r = threadIdx.x; r < g.Ns; r += blockDim.x) h += (double)tb.mult[r] * row_value(G, d, tb, g, r, 0);
        h = 2.0 * h;
        if (threadIdx.x == 0) {
            Desc<double> e;
            make_desc(w1 + w2, w2 - w1, 0.0, 2, 0, tb, g, e);
            T f = T(0.0);
            if (g.nc == 2) f = row_value(G, e, tb, g, 0, 0) + 3.0 * row_value(G, e, tb, g, 0, 1);
            else for (int c = 0; c < 4; ++c) f += row_value(G, e, tb, g, 0, c);
            h -= f;
        }
        H[sg] = h;
    }
    block_sum<T, 2>(H, red);
    if (threadIdx.x == 0) {
        T acc = T(0.0);
        acc += H[0] / (lam + interp_odd(w, tb.invh, g.N, gam, lam));
        acc += H[1] / (-lam + interp_odd(w, tb.invh, g.N, gam, -lam));
        dgam[n] = -acc / (2.0 * kPi);
    }
}

template <typename T>
__global__ void k_sigma_rhs(Geo g, Tabs tb, const double* __restrict__ w, const T* __restrict__ gam,
                            const T* __restrict__ G, double lam, T* __restrict__ dgam) {
    sigma_rhs_block<T>(g, tb, w, gam, G, lam, dgam, blockIdx.x);
}

// Projected products of the three channels (hand-derived from the Pauli algebra):
// SU2 (d = Gamma^00, s = Gamma^zz) and XYZ (0, x, y, z).
template <typename T, int NC>
__device__ __forceinline__ void s_product(const T* A, const T* B, T* o) {
    if (NC == 2) {
        o[0] = A[0] * B[0] + (T)3 * A[1] * B[1];
        o[1] = A[0] * B[1] + A[1] * B[0] - (T)2 * A[1] * B[1];
    } else {
        o[0] = A[0] * B[0] + A[1] * B[1] + A[2] * B[2] + A[3] * B[3];
        o[1] = A[0] * B[1] + A[1] * B[0] - (A[2] * B[3] + A[3] * B[2]);
        o[2] = A[0] * B[2] + A[2] * B[0] - (A[1] * B[3] + A[3] * B[1]);
        o[3] = A[0] * B[3] + A[3] * B[0] - (A[1] * B[2] + A[2] * B[1]);
    }
}
template <typename T, int NC>
__device__ __forceinline__ void u_product(const T* A, const T* B, T* o) {
    if (NC == 2) {
        o[0] = A[0] * B[0] + (T)3 * A[1] * B[1];
        o[1] = A[0] * B[1] + A[1] * B[0] + (T)2 * A[1] * B[1];
    } else {
        o[0] = A[0] * B[0] + A[1] * B[1] + A[2] * B[2] + A[3] * B[3];
        o[1] = A[0] * B[1] + A[1] * B[0] + (A[2] * B[3] + A[3] * B[2]);
        o[2] = A[0] * B[2] + A[2] * B[0] + (A[1] * B[3] + A[3] * B[1]);
        o[3] = A[0] * B[3] + A[3] * B[0] + (A[1] * B[2] + A[2] * B[1]);
    }
}
// a * b + c as one fused multiply-add (for dual numbers: the same value, tangents by the
// product rule)
__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
template <int P>
__device__ __forceinline__ Dual<P> fmadd(const Dual<P>& a, const Dual<P>& b, const Dual<P>& c) { return a * b + c; }
template <int P>
__device__ __forceinline__ Dual<P> fmadd(const Dual<P>& a, double b, const Dual<P>& c) { return a * b + c; }

// acc += s_product(A, B) (SGN = -1) or u_product(A, B) (SGN = +1) as chains of fused
// multiply-adds into the accumulators.
template <typename T, int NC, int SGN>
__device__ __forceinline__ void su_product_acc(const T* A, const T* B, T* acc) {
    if (NC == 2) {
        const T t = A[1] * B[1];
        acc[0] = fmadd(A[0], B[0], acc[0]);
        acc[0] = fmadd(t, (T)3, acc[0]);
        acc[1] = fmadd(A[0], B[1], acc[1]);
        acc[1] = fmadd(A[1], B[0], acc[1]);
        acc[1] = fmadd(t, (T)(2 * SGN), acc[1]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[0] = fmadd(A[k], B[k], acc[0]);
#pragma unroll
        for (int c = 1; c < 4; ++c) {
            const int p = c == 1 ? 2 : 1, q = c == 3 ? 2 : 3;   // the two other spin components
            acc[c] = fmadd(A[0], B[c], acc[c]);
            acc[c] = fmadd(A[c], B[0], acc[c]);
            acc[c] = fmadd(SGN > 0 ? A[p] : -A[p], B[q], acc[c]);
            acc[c] = fmadd(SGN > 0 ? A[q] : -A[q], B[p], acc[c]);
        }
    }
}

// On-site factor sum_k s(k, c) C_k with s = -1 iff k and c are distinct spin components.
template <typename T, int NC>
__device__ __forceinline__ T onsite_factor(const T* C, int c) {
    if (NC == 2) return c == 0 ? C[0] + (T)3 * C[1] : C[0] - C[1];
    T acc = C[0];
#pragma unroll
    for (int k = 1; k < 4; ++k) acc += (c == 0 || k == c) ? C[k] : -C[k];
    return acc;
}

template <typename T>
struct ShPtrs {
    T* acc;
    T* part;
    Desc<typename WeightOf<T>::type>* desc;
    T* rows;
    T* onrow;
    T* wq;
};

template <typename T, int NC>
__device__ __forceinline__ ShPtrs<T> carve(unsigned char* raw, const Geo& g, const Tabs& tb) {
    ShPtrs<T> p;
    size_t off = 0;
    auto take = [&](size_t bytes) { unsigned char* q = raw + off; off += (bytes + 15) & ~size_t(15); return q; };
    p.desc = (Desc<typename WeightOf<T>::type>*)take(sizeof(Desc<typename WeightOf<T>::type>) * kQC * 4);
    p.acc = (T*)take(sizeof(T) * g.Ns * NC);
    p.part = (T*)take(sizeof(T) * tb.nprod);
    p.rows = (T*)take(sizeof(T) * kQC * 2 * g.Ns * NC);
    p.onrow = (T*)take(sizeof(T) * kQC * 2 * NC);
    p.wq = (T*)take(sizeof(T) * kQC);
    return p;
}

// Vertex arguments of one integration node (Eq. frg:flowexplicit:2particle):
// row 0 / 1 of the s channel: (s, w1'-x, x-w2') and (s, x-w1, x-w2);
// t channel: (w1+x, t, w1'-x), (x+w2', t, x-w2), on-site (w2'+x, w2-x, -t), (w1+x, x-w1', -t);
// u channel: (w1+x, x-w2', u) and (w1'+x, w2-x, u).
template <typename F = double>
__device__ __forceinline__ void node_args(int ch, int rw, F x, F s, F t, F u, F w1p, F w2p, F w1, F w2, F& a, F& b, F& c) {
    if (ch == 0) {
        if (rw == 0) { a = s; b = w1p - x; c = x - w2p; }
        else { a = s; b = x - w1; c = x - w2; }
    } else if (ch == 1) {
        if (rw == 0) { a = w1 + x; b = t; c = w1p - x; }
        else if (rw == 1) { a = x + w2p; b = t; c = x - w2; }
        else if (rw == 2) { a = w2p + x; b = w2 - x; c = -t; }
        else { a = w1 + x; b = x - w1p; c = -t; }
    } else {
        if (rw == 0) { a = w1 + x; b = x - w2p; c = u; }
        else { a = w1p + x; b = w2 - x; c = u; }
    }
}

template <typename T, int NC>
__global__ void __launch_bounds__(kThreads, std::is_same<T, double>::value ? 6 : 1) k_gamma_rhs(Geo g, Tabs tb, const double* __restrict__ w,
                                                        const T* __restrict__ G, const double* __restrict__ nx,
                                                        const T* __restrict__ nW, const int* __restrict__ ncount,
                                                        T* __restrict__ dG, int p0) {
    extern __shared__ __align__(16) unsigned char smem[];
    ShPtrs<T> sh = carve<T, NC>(smem, g, tb);
    const int tid = threadIdx.x;
    const int ti = blockIdx.x % g.N;
    const int p = p0 + (int)(blockIdx.x / g.N);   // stored pairs p0, p0 + 1, ...: one CTA per triple
    int si = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
    while ((si + 1) * (si + 2) / 2 <= p) ++si;
    while (si * (si + 1) / 2 > p) --si;
    const int ui = p - si * (si + 1) / 2;
    const double s = w[si], t = w[ti], u = w[ui];
    const double w1p = (s + t + u) / 2, w2p = (s - t - u) / 2, w1 = (s - t + u) / 2, w2 = (s + t - u) / 2;
    const int row = g.Ns * NC;

    for (int o = tid; o < row; o += blockDim.x) sh.acc[o] = (T)0;
    for (int o = tid; o < tb.nprod; o += blockDim.x) sh.part[o] = (T)0;
    // per-site products: thread (site my_r, node group my_g) takes every NG-th node of a block
    // and keeps its partial sums in registers for the whole channel
    const bool site_reg = g.Ns <= (int)blockDim.x;
    const int NG = site_reg ? min((int)blockDim.x / g.Ns, kQC) : 1;
    const int my_r = tid % g.Ns, my_g = tid / g.Ns;
    const bool site_on = site_reg && my_g < NG;
    // FP64: lattice-sum integrals of the products tid + k blockDim held in registers across the
    // t channel when every thread owns at most kPR products
    constexpr int kPR = 8;
    constexpr bool kRegT = std::is_same<T, double>::value;
    const bool preg = kRegT && tb.nprod <= kPR * (int)blockDim.x;
    double pacc[kPR];
#pragma unroll
    for (int k = 0; k < kPR; ++k) pacc[k] = 0.0;

    for (int ch = 0; ch < 3; ++ch) {
        const int vi = ch == 0 ? si : (ch == 1 ? ti : ui);
        const int cidx = ch * g.N + vi;
        const int nq = ncount[cidx];
        const double* X = nx + (size_t)cidx * g.nmax;
        const T* Wp = nW + (size_t)cidx * g.nmax;
        const int nrow = ch == 1 ? 4 : 2;
        T racc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) racc[c] = (T)0;
        for (int q0 = 0; q0 < nq; q0 += kQC) {
            const int qn = min(kQC, nq - q0);
            __syncthreads();
            // phase 1: lookup descriptors of every row at every node of this block
            for (int idx = tid; idx < qn * nrow; idx += blockDim.x) {
                const int q = idx / nrow, rw = idx % nrow;
                const double x = X[q0 + q];
                double a, b, c;
                node_args(ch, rw, x, s, t, u, w1p, w2p, w1, w2, a, b, c);
                const int exs = ch == 0 ? 0 : (ch == 2 ? 2 : (rw < 2 ? 1 : 2));
                Desc<typename WeightOf<T>::type>& d = sh.desc[q * 4 + rw];
                if (rw == 0) sh.wq[q] = Wp[q0 + q];
                if constexpr (std::is_same<T, double>::value) {
                    // FP64: the node weight goes into the corner weights of its rows
                    make_desc<double, true>(a, b, c, exs, vi, tb, g, d, (rw == 0 || rw == 3) ? Wp[q0 + q] : 1.0);
                } else {
                    make_desc(a, b, c, exs, vi, tb, g, d);
                }
            }
            __syncthreads();
            // phase 2: interpolated rows over all irreducible sites (and the on-site rows); the
            // first row of every node (and the second on-site row) carries the node weight
            constexpr bool kWeighted = std::is_same<T, double>::value;   // already in the corners
            {
                const int nfull = qn * 2 * row;
                int q = tid / (2 * row), rem = tid % (2 * row);
                int rw = rem / row, e = rem % row;
                for (int idx = tid; idx < nfull; idx += blockDim.x) {
                    const int r = e / NC, c = e % NC;
                    T v = row_value(G, sh.desc[q * 4 + rw], tb, g, r, c);
                    if (!kWeighted && rw == 0) v *= sh.wq[q];
                    sh.rows[(q * 2 + rw) * row + e] = v;
                    e += blockDim.x;
                    while (e >= row) { e -= row; if (++rw == 2) { rw = 0; ++q; } }
                }
                if (ch == 1) {
                    // on-site rows C (rr = 0) and D (rr = 1), stored as their on-site factors
                    // F_c = sum_k s(k, c) X_k; a site whose on-site pair carries the component
                    // permutation pi reads F_pi(c) of C (pi fixes the density component)
                    for (int j = tid; j < qn * 2; j += blockDim.x) {
                        const int qq = j >> 1, rr = j & 1;
                        T v[NC];
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            v[c] = row_value(G, sh.desc[qq * 4 + 2 + rr], tb, g, 0, c);
                            if (!kWeighted && rr == 1) v[c] *= sh.wq[qq];
                        }
#pragma unroll
                        for (int c = 0; c < NC; ++c) sh.onrow[(qq * 2 + rr) * NC + c] = onsite_factor<T, NC>(v, c);
                    }
                }
            }
            __syncthreads();
            // phase 3: products
            if (ch != 1) {
                if (site_on)
                    for (int q = my_g; q < qn; q += NG) {
                        const T* A = sh.rows + (q * 2) * row + my_r * NC;
                        const T* B = sh.rows + (q * 2 + 1) * row + my_r * NC;
                        if (ch == 0) su_product_acc<T, NC, -1>(A, B, racc); else su_product_acc<T, NC, 1>(A, B, racc);
                    }
                for (int r = site_reg ? g.Ns : tid; r < g.Ns; r += blockDim.x) {
                    T accl[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c) accl[c] = (T)0;
                    for (int q = 0; q < qn; ++q) {
                        const T* A = sh.rows + (q * 2) * row + r * NC;
                        const T* B = sh.rows + (q * 2 + 1) * row + r * NC;
                        if (ch == 0) su_product_acc<T, NC, -1>(A, B, accl); else su_product_acc<T, NC, 1>(A, B, accl);
                    }
#pragma unroll
                    for (int c = 0; c < NC; ++c) sh.acc[r * NC + c] += accl[c];
                }
            } else {
                // lattice sum: every distinct product (row A entry, row B entry) integrated over
                // the nodes of this block; each product is owned by one thread across blocks
                if constexpr (kRegT) {
                    if (preg) {
                        int ia[kPR], ib[kPR];
#pragma unroll
                        for (int k = 0; k < kPR; ++k) {
                            const int o = tid + k * (int)blockDim.x;
                            const int2 pr = o < tb.nprod ? tb.prod[o] : make_int2(-1, 0);
                            ia[k] = pr.x;
                            ib[k] = pr.y;
                        }
#pragma unroll 1
                        for (int q = 0; q < qn; ++q) {
                            const double* Ar = reinterpret_cast<const double*>(sh.rows) + (q * 2) * row;
                            const double* Br = Ar + row;
#pragma unroll
                            for (int k = 0; k < kPR; ++k)
                                if (ia[k] >= 0) pacc[k] = fma(Ar[ia[k]], Br[ib[k]], pacc[k]);
                        }
                    }
                }
                for (int o = preg ? tb.nprod : tid; o < tb.nprod; o += blockDim.x) {
                    const int2 pr = tb.prod[o];
                    T a = (T)0;
                    for (int q = 0; q < qn; ++q)
                        a += sh.rows[(q * 2) * row + pr.x] * sh.rows[(q * 2 + 1) * row + pr.y];
                    sh.part[o] += a;
                }
                // on-site terms
                if (site_on) {
                    const int pon = tb.onsite_perm[my_r];
                    for (int q = my_g; q < qn; q += NG) {
                        const T* A = sh.rows + (q * 2) * row + my_r * NC;
                        const T* B = sh.rows + (q * 2 + 1) * row + my_r * NC;
                        const T* FC = sh.onrow + (q * 2) * NC;
                        const T* FD = sh.onrow + (q * 2 + 1) * NC;
#pragma unroll
                        for (int c = 0; c < NC; ++c)
                            racc[c] = fmadd(A[c], FC[perm_of(pon, c)], fmadd(FD[c], B[c], racc[c]));
                    }
                }
                for (int r = site_reg ? g.Ns : tid; r < g.Ns; r += blockDim.x) {
                    const int pon = tb.onsite_perm[r];
                    T accl[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c) accl[c] = (T)0;
                    for (int q = 0; q < qn; ++q) {
                        const T* A = sh.rows + (q * 2) * row + r * NC;
                        const T* B = sh.rows + (q * 2 + 1) * row + r * NC;
                        const T* FC = sh.onrow + (q * 2) * NC;
                        const T* FD = sh.onrow + (q * 2 + 1) * NC;
#pragma unroll
                        for (int c = 0; c < NC; ++c)
                            accl[c] = fmadd(A[c], FC[perm_of(pon, c)], fmadd(FD[c], B[c], accl[c]));
                    }
#pragma unroll
                    for (int c = 0; c < NC; ++c) sh.acc[r * NC + c] += accl[c];
                }
            }
        }
        if (site_reg) {
            // combine the node groups' register partials in a fixed order (scratch: the rows)
            __syncthreads();
            T* scr = sh.rows;
            if (site_on)
#pragma unroll
                for (int c = 0; c < NC; ++c) scr[(my_g * NC + c) * g.Ns + my_r] = racc[c];
            __syncthreads();
            for (int o = tid; o < row; o += blockDim.x) {
                const int r = o / NC, c = o % NC;
                T a = (T)0;
                for (int k = 0; k < NG; ++k) a += scr[(k * NC + c) * g.Ns + r];
                sh.acc[o] += a;
            }
        }
    }
    if (preg)
#pragma unroll
        for (int k = 0; k < kPR; ++k) {
            const int o = tid + k * (int)blockDim.x;
            if (o < tb.nprod) sh.part[o] = (T)pacc[k];
        }
    __syncthreads();
    for (int o = tid; o < row; o += blockDim.x) {
        const int r = o / NC, c = o % NC;
        T a = (T)0;
        for (int k = tb.gath_off[o]; k < tb.gath_off[o + 1]; ++k) a += sh.part[tb.gath_idx[k]];
        const T v = sh.acc[o] - 2.0 * a;
        dG[((size_t)(p * g.N + ti) * NC + c) * g.Ns + r] = v;
    }
}


// ----------------------------------------------------------------------------- FP32 vertex flow

constexpr int kQF = 32;   // integration nodes per shared-memory block (FP32 kernel)

template <int NC, bool DENSE>
struct ShF {
    DescF* desc;
    float* rows;
    float* onrow;
    float* wq;
    float* acc;
    float* cacc;
};

__host__ __device__ inline size_t rnd16(size_t b) { return (b + 15) & ~size_t(15); }

// Tensor-core lattice sum (SU2, padded sites nsp <= 64): per triple and component c the dense
// contraction C_c[rA][rB] = sum_q A_q[c][rA] B_q[c][rB] as tcgen05 MMAs with M = 64 (rA),
// N = NB (rB), K = 8 nodes, in 3xTF32 (A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulation in
// TMEM).  For nsp <= 32 both components share one MMA ("packed": A rows c * 32 + rA, B rows
// c * Np + rB; only the c = c' blocks of the product are read back).
constexpr int kQT = 16;   // t-channel nodes per block on the tensor-core path (two K-steps)

struct TcShape {
    int packed, G, Np, NB, ncols;   // MMA groups G (1 packed, 2 one per component), N per MMA
    int tileA, tileB, kbytes;       // bytes of an A / B tile (K = 8) and of one K-step's tiles
};

__host__ __device__ inline TcShape tc_shape(int nsp) {
    TcShape t;
    t.packed = nsp <= 32;
    t.Np = (nsp + 7) & ~7;
    t.NB = t.packed ? 2 * t.Np : t.Np;
    t.G = t.packed ? 1 : 2;
    t.ncols = 32;
    while (t.ncols < t.G * t.NB) t.ncols *= 2;
    t.tileA = 64 * 32;
    t.tileB = t.NB * 32;
    t.kbytes = t.G * 2 * (t.tileA + t.tileB);
    return t;
}

__host__ __device__ inline bool tc_supported(int nc, int nsp, bool dense) { return nc == 2 && dense && nsp <= 64; }

__host__ __device__ inline size_t f32_smem_bytes(int Ns, int nsp, int nc, int nprod, bool dense, bool tc = false) {
    const size_t rowp = (size_t)nc * nsp;
    size_t rows = sizeof(float) * kQF * 2 * rowp;
    if (tc) rows = rows > (size_t)(kQT / 8) * tc_shape(nsp).kbytes ? rows : (size_t)(kQT / 8) * tc_shape(nsp).kbytes;
    return rnd16(sizeof(DescF) * kQF * 4) + rnd16(rows) + rnd16(sizeof(float) * kQF * 2 * nc) +
           rnd16(sizeof(float) * kQF) + rnd16(sizeof(float) * Ns * nc) +
           rnd16(sizeof(float) * (dense ? (size_t)nc * nsp * nsp : (size_t)nprod));
}

// Tensor-memory state of a CTA on the tensor-core path.
struct TcCta {
    uint32_t tmem;      // accumulator base address (lane 0, first column)
    uint64_t* mbar;     // MMA completion barrier
    uint32_t ncommit;   // commits so far (the barrier's completed phases)
    int* fail;          // set when a completion wait gives up
};

// t channel of one stored triple on the tensor-core path: node blocks of kQT nodes; the
// interpolated rows A (weighted) and B go to shared memory as TF32 hi / lo tiles; one thread
// issues the 3xTF32 MMAs of the block (accumulating C in TMEM across the channel) while all
// threads add the on-site terms; at the end C is read back into cacc for the table gather.
template <typename Sh>
__device__ void t_channel_tc(const Geo& g, const Tabs& tb, const float* __restrict__ Gf, const float* __restrict__ Gs,
                             const float* __restrict__ X, const float* __restrict__ Wp, const int nq, const int vi,
                             const float s, const float t, const float u, const float w1p, const float w2p,
                             const float w1, const float w2, Sh& sh, float (&racc)[2], const bool site_on,
                             const int my_r, const int my_g, const int NG, TcCta& tcs) {
    constexpr int NC = 2;
    const int tid = threadIdx.x;
    const int nsp = g.nsp, nsp4 = nsp >> 2, rowp = NC * nsp;
    const TcShape ts = tc_shape(nsp);
    unsigned char* tiles = reinterpret_cast<unsigned char*>(sh.rows);
    const uint32_t tiles_s = tc::smem_addr(tiles);
    const uint32_t idesc = tc::idesc_tf32(64, ts.NB);
    constexpr long kWait = 1L << 22;
    __syncthreads();   // the previous channel's scratch reads of this region are done
    // zero every tile once: padding rows (sites >= nsp, unused M rows) stay zero
    for (int i = tid; i < (kQT / 8) * ts.kbytes / 16; i += blockDim.x)
        reinterpret_cast<float4*>(tiles)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    bool started = false;
    for (int q0 = 0; q0 < nq; q0 += kQT) {
        const int qn = min(kQT, nq - q0), qpad = (qn + 7) & ~7;
        __syncthreads();
        for (int idx = tid; idx < qn * 4; idx += blockDim.x) {
            const int q = idx / 4, rw = idx % 4;
            const float x = X[q0 + q];
            float a, b, c;
            node_args<float>(1, rw, x, s, t, u, w1p, w2p, w1, w2, a, b, c);
            DescF dl;
            make_desc4(a, b, c, rw < 2 ? 1 : 2, vi, tb, g, rowp, dl);
            store_desc4(&sh.desc[q * 4 + rw], dl, tid & 31);
            if (rw == 0) sh.wq[q] = Wp[q0 + q];
        }
        // the previous block's MMAs must have read their tiles before they are rewritten
        if (started && !tc::mbar_wait(tcs.mbar, (tcs.ncommit - 1) & 1, kWait) && tid == 0) atomicOr(tcs.fail, 1);
        __syncthreads();
        // item = (4-node group, row, component, 4 sites); the four lanes of a quad take the four
        // nodes of a group, interpolate 4 sites each, and transpose through shuffles so that
        // each lane stores one site's 4 consecutive nodes: a 16-byte row of a core matrix
        const int nitems = qpad * 2 * NC * nsp4;   // a multiple of 4: quads never straddle the end
        const int ql = tid & 3;
        for (int base = 0; base < nitems; base += blockDim.x) {
            const int it = base + tid;
            const bool act = it < nitems;
            int rest = it >> 2;
            const int r4 = rest % nsp4;
            rest /= nsp4;
            const int c = rest % NC;
            rest /= NC;
            const int rw = rest & 1, q = 4 * (rest >> 1) + ql;
            float vv[4] = {0.f, 0.f, 0.f, 0.f};
            if (act && q < qn) {
                const DescF& d = sh.desc[q * 4 + rw];
                const float* gb = (d.swap ? Gs : Gf) + c * nsp + 4 * r4;
                const int4 ov = *reinterpret_cast<const int4*>(d.off);
                const float4 wv = c == 0 ? *reinterpret_cast<const float4*>(d.wd) : *reinterpret_cast<const float4*>(d.ws);
                const float4 g0 = __ldg(reinterpret_cast<const float4*>(gb + ov.x));
                const float4 g1 = __ldg(reinterpret_cast<const float4*>(gb + ov.y));
                const float4 g2 = __ldg(reinterpret_cast<const float4*>(gb + ov.z));
                const float4 g3 = __ldg(reinterpret_cast<const float4*>(gb + ov.w));
                vv[0] = wv.x * g0.x + wv.y * g1.x + wv.z * g2.x + wv.w * g3.x;
                vv[1] = wv.x * g0.y + wv.y * g1.y + wv.z * g2.y + wv.w * g3.y;
                vv[2] = wv.x * g0.z + wv.y * g1.z + wv.z * g2.z + wv.w * g3.z;
                vv[3] = wv.x * g0.w + wv.y * g1.w + wv.z * g2.w + wv.w * g3.w;
                if (rw == 0) {
                    const float wq = sh.wq[q];
#pragma unroll
                    for (int j = 0; j < 4; ++j) vv[j] *= wq;
                }
            }
            // 4 x 4 transpose in the quad: round k sends vv[(ql + k) & 3] and receives site ql of
            // node (ql - k) & 3
            float uu[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int si_ = (ql + k) & 3, src = (ql - k) & 3;
                const float send = si_ == 0 ? vv[0] : (si_ == 1 ? vv[1] : (si_ == 2 ? vv[2] : vv[3]));
                const float got = __shfl_sync(0xffffffffu, send, (tid & 31 & ~3) | src);
                if (src == 0) uu[0] = got;
                else if (src == 1) uu[1] = got;
                else if (src == 2) uu[2] = got;
                else uu[3] = got;
            }
            if (act) {
                const int gi = ts.packed ? 0 : c;
                const int q0g = q & ~3;   // first node of the group
                unsigned char* kb = tiles + (q0g >> 3) * ts.kbytes + gi * 2 * (ts.tileA + ts.tileB);
                unsigned char* hi = rw == 0 ? kb : kb + 2 * ts.tileA;
                unsigned char* lo = hi + (rw == 0 ? ts.tileA : ts.tileB);
                const int r = (ts.packed ? c * (rw == 0 ? 32 : ts.Np) : 0) + 4 * r4 + ql;
                float4 h, l;
                h.x = tc::tf32_rna(uu[0]); l.x = tc::tf32_rna(uu[0] - h.x);
                h.y = tc::tf32_rna(uu[1]); l.y = tc::tf32_rna(uu[1] - h.y);
                h.z = tc::tf32_rna(uu[2]); l.z = tc::tf32_rna(uu[2] - h.z);
                h.w = tc::tf32_rna(uu[3]); l.w = tc::tf32_rna(uu[3] - h.w);
                const uint32_t o = tc::tile_off(r, q0g & 7);
                *reinterpret_cast<float4*>(hi + o) = h;
                *reinterpret_cast<float4*>(lo + o) = l;
            }
        }
        for (int j = tid; j < qn * 2 * NC; j += blockDim.x) {
            const int qq = j / (2 * NC), rr = (j / NC) % 2, c = j % NC;
            const DescF& d = sh.desc[qq * 4 + 2 + rr];
            const float* base = Gf + c * nsp;   // the on-site pair is its own exchange
            const float* wgt = c == 0 ? d.wd : d.ws;
            float v = 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) v += wgt[k] * base[d.off[k]];
            if (rr == 1) v *= sh.wq[qq];
            sh.onrow[(qq * 2 + rr) * NC + c] = v;
        }
        tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            for (int ks = 0; ks < qpad / 8; ++ks)
                for (int gi = 0; gi < ts.G; ++gi) {
                    const uint32_t kb = tiles_s + ks * ts.kbytes + gi * 2 * (ts.tileA + ts.tileB);
                    const uint64_t ah = tc::smem_desc(kb), al = tc::smem_desc(kb + ts.tileA);
                    const uint64_t bh = tc::smem_desc(kb + 2 * ts.tileA), bl = tc::smem_desc(kb + 2 * ts.tileA + ts.tileB);
                    const uint32_t d = tcs.tmem + gi * ts.NB;
                    tc::mma_tf32(d, ah, bh, idesc, started || ks > 0);
                    tc::mma_tf32(d, ah, bl, idesc, true);
                    tc::mma_tf32(d, al, bh, idesc, true);
                }
            tc::mma_commit(tcs.mbar);
        }
        tcs.ncommit++;
        started = true;
        // on-site terms of this block (rows read back as hi + lo) while the MMAs run
        if (site_on) {
            const int r = my_r;
            const int pon = tb.onsite_perm[r];
            for (int q = my_g; q < qn; q += NG) {
                const unsigned char* kb = tiles + (q >> 3) * ts.kbytes;
                float A[NC], B[NC], Cp[NC], D[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const unsigned char* gb = kb + (ts.packed ? 0 : c) * 2 * (ts.tileA + ts.tileB);
                    const uint32_t oa = tc::tile_off((ts.packed ? c * 32 : 0) + r, q & 7);
                    const uint32_t ob = tc::tile_off((ts.packed ? c * ts.Np : 0) + r, q & 7);
                    A[c] = *reinterpret_cast<const float*>(gb + oa) + *reinterpret_cast<const float*>(gb + ts.tileA + oa);
                    B[c] = *reinterpret_cast<const float*>(gb + 2 * ts.tileA + ob) +
                           *reinterpret_cast<const float*>(gb + 2 * ts.tileA + ts.tileB + ob);
                    Cp[c] = sh.onrow[(q * 2) * NC + perm_of(pon, c)];
                    D[c] = sh.onrow[(q * 2 + 1) * NC + c];
                }
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    racc[c] = fmadd(A[c], onsite_factor<float, NC>(Cp, c), fmadd(onsite_factor<float, NC>(D, c), B[c], racc[c]));
            }
        }
    }
    if (!started) return;   // no node: C stays zero
    if (!tc::mbar_wait(tcs.mbar, (tcs.ncommit - 1) & 1, kWait) && tid == 0) atomicOr(tcs.fail, 1);
    tc::fence_after_sync();
    // read C back: warp w holds accumulator rows 16 w .. 16 w + 15 in its lanes 0..15
    const int warp = tid >> 5, lane = tid & 31;
    if (warp < 4) {
        const int m = 16 * warp + lane;
        for (int j = 0; j < ts.G * ts.NB / 8; ++j) {
            float v[8];
            tc::tmem_ld8(tcs.tmem + ((uint32_t)(32 * warp) << 16) + 8 * j, v);
            if (lane < 16) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int col = 8 * j + i, gi = col / ts.NB, n = col % ts.NB;
                    int c, rA, rB;
                    if (ts.packed) {
                        c = m / 32; rA = m % 32;
                        if (n / ts.Np != c) continue;
                        rB = n % ts.Np;
                    } else {
                        c = gi; rA = m; rB = n;
                    }
                    if (rA < nsp && rB < nsp) sh.cacc[c * nsp * nsp + rA * nsp + rB] = v[i];
                }
            }
        }
    }
    tc::fence_before_sync();
}

// FP32-mixed vertex flow: the same equations as k_gamma_rhs with FP32 rows, products and
// accumulation (descriptor decisions and node positions stay FP64).  Rows are interpolated
// four padded sites at a time from the FP32 shadow (Gs: the same shadow with the exchanged
// pair stored in place, for lookups whose arguments exchange the two sites).  With DENSE
// (SU2), the lattice sum is the per-triple contraction C[c][rA][rB] = sum_q A_q B_q in 4x4
// register tiles, gathered through the table at the end.
template <int NC, bool DENSE, bool TC = false>
__device__ void gamma_rhs_f32_triple(const Geo& g, const Tabs& tb, const float* __restrict__ Gf,
                                     const float* __restrict__ Gs, const float* __restrict__ nx,
                                     const float* __restrict__ nW, const int* __restrict__ ncount,
                                     double* __restrict__ dG, const int p, const int ti, unsigned char* smem,
                                     const int qc, TcCta* tcs = nullptr) {
    static_assert(!TC || (NC == 2 && DENSE), "tensor-core lattice sum: SU2 dense contraction only");
    const int nsp = g.nsp, nsp4 = nsp >> 2, rowp = NC * nsp;
    // n / nsp4 as __umulhi(n, div4) with div4 = ceil(2^32 / nsp4): exact for n nsp4 < 2^32
    // (nsp4 = 1 is taken separately: its multiplier does not fit 32 bits)
    const unsigned div4 = g.div4;
    ShF<NC, DENSE> sh;
    {
        size_t off = 0;
        auto take = [&](size_t bytes) { unsigned char* q = smem + off; off += rnd16(bytes); return q; };
        sh.desc = (DescF*)take(sizeof(DescF) * kQF * 4);
        size_t rows_bytes = sizeof(float) * kQF * 2 * rowp;
        if (TC) rows_bytes = max(rows_bytes, (size_t)(kQT / 8) * tc_shape(nsp).kbytes);
        sh.rows = (float*)take(rows_bytes);
        sh.onrow = (float*)take(sizeof(float) * kQF * 2 * NC);
        sh.wq = (float*)take(sizeof(float) * kQF);
        sh.acc = (float*)take(sizeof(float) * g.Ns * NC);
        sh.cacc = (float*)take(sizeof(float) * (DENSE ? NC * nsp * nsp : tb.nprod));
    }
    const int tid = threadIdx.x;
    int si = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);   // guess, corrected below
    while ((si + 1) * (si + 2) / 2 <= p) ++si;
    while (si * (si + 1) / 2 > p) --si;
    const int ui = p - si * (si + 1) / 2;
    const float* w = tb.wf;
    __syncthreads();   // shared memory of a previous triple (persistent callers) is consumed
    // frequencies and integration nodes in FP32 (the descriptors of this kernel are FP32)
    const float s = w[si], t = w[ti], u = w[ui];
    const float w1p = (s + t + u) * 0.5f, w2p = (s - t - u) * 0.5f, w1 = (s - t + u) * 0.5f, w2 = (s + t - u) * 0.5f;
    const int ncacc = DENSE ? NC * nsp * nsp : tb.nprod;
    for (int o = tid; o < g.Ns * NC; o += blockDim.x) sh.acc[o] = 0.0f;
    for (int o = tid; o < ncacc; o += blockDim.x) sh.cacc[o] = 0.0f;

    // work split of the per-site and per-tile products: thread (r, group) takes every NG-th
    // node of a block and keeps its partial sums in registers for the whole channel
    const bool site_reg = g.Ns <= (int)blockDim.x;
    const int NG = site_reg ? (int)blockDim.x / g.Ns : 1;
    const int my_r = tid % g.Ns, my_g = tid / g.Ns;
    const bool site_on = site_reg && my_g < NG;
    const int ntile = NC * nsp4 * nsp4;
    const size_t site_part = site_reg ? (size_t)NG * g.Ns * NC : 0;   // scratch floats of the site partials
    const bool tile_reg = DENSE && !TC && ntile <= (int)blockDim.x &&
                          site_part + (size_t)((int)blockDim.x / ntile) * ntile * 16 <= (size_t)kQF * 2 * rowp;
    const int TG = tile_reg ? (int)blockDim.x / ntile : 1;
    const int my_tile = tid % ntile, my_tg = tid / ntile;
    const bool tile_on = tile_reg && my_tg < TG;
    for (int ch = 0; ch < 3; ++ch) {
        const int vi = ch == 0 ? si : (ch == 1 ? ti : ui);
        float racc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) racc[c] = 0.0f;
        float a4[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) a4[i][j] = 0.0f;
        const int cidx = ch * g.N + vi;
        const int nq = ncount[cidx];
        const float* X = nx + (size_t)cidx * g.nmax;
        const float* Wp = nW + (size_t)cidx * g.nmax;
        const int nrow = ch == 1 ? 4 : 2;
        if constexpr (TC) {
            if (ch == 1)
                t_channel_tc(g, tb, Gf, Gs, X, Wp, nq, vi, s, t, u, w1p, w2p, w1, w2, sh, racc, site_on, my_r, my_g, NG, *tcs);
        }
        for (int q0 = 0; q0 < ((TC && ch == 1) ? 0 : nq); q0 += qc) {
            const int qn = min(qc, nq - q0);
            __syncthreads();
            for (int idx = tid; idx < qn * nrow; idx += blockDim.x) {
                const int q = idx / nrow, rw = idx % nrow;
                const float x = X[q0 + q];
                float a, b, c;
                node_args<float>(ch, rw, x, s, t, u, w1p, w2p, w1, w2, a, b, c);
                const int exs = ch == 0 ? 0 : (ch == 2 ? 2 : (rw < 2 ? 1 : 2));
                DescF dl;
                make_desc4(a, b, c, exs, vi, tb, g, rowp, dl);
                if (rw == 0 || rw == 3) {   // the node weight goes into the corner weights
                    const float wn = Wp[q0 + q];
#pragma unroll
                    for (int k = 0; k < 4; ++k) { dl.wd[k] *= wn; dl.ws[k] *= wn; }
                }
                store_desc4(&sh.desc[q * 4 + rw], dl, tid & 31);
            }
            __syncthreads();
            // rows: four padded sites per item; row 0 (and on-site row 1) carry the node weight
            const int nitems = qn * 2 * NC * nsp4;
            for (int it = tid; it < nitems; it += blockDim.x) {
                const int t2f = nsp4 > 1 ? (int)__umulhi((unsigned)it, div4) : it;   // it / nsp4
                const int r4 = it - t2f * nsp4;
                int t2 = t2f;
                const int c = t2 % NC;
                t2 /= NC;
                const int rw = t2 & 1, q = t2 >> 1;
                const DescF& d = sh.desc[q * 4 + rw];
                const float* base = (d.swap ? Gs : Gf) + c * nsp + 4 * r4;
                const int4 ov = *reinterpret_cast<const int4*>(d.off);
                const float4 wv = c == 0 ? *reinterpret_cast<const float4*>(d.wd) : *reinterpret_cast<const float4*>(d.ws);
                const float4 g0 = __ldg(reinterpret_cast<const float4*>(base + ov.x));
                const float4 g1 = __ldg(reinterpret_cast<const float4*>(base + ov.y));
                const float4 g2 = __ldg(reinterpret_cast<const float4*>(base + ov.z));
                const float4 g3 = __ldg(reinterpret_cast<const float4*>(base + ov.w));
                float4 v;
                v.x = wv.x * g0.x + wv.y * g1.x + wv.z * g2.x + wv.w * g3.x;
                v.y = wv.x * g0.y + wv.y * g1.y + wv.z * g2.y + wv.w * g3.y;
                v.z = wv.x * g0.z + wv.y * g1.z + wv.z * g2.z + wv.w * g3.z;
                v.w = wv.x * g0.w + wv.y * g1.w + wv.z * g2.w + wv.w * g3.w;
                *reinterpret_cast<float4*>(sh.rows + (q * 2 + rw) * rowp + c * nsp + 4 * r4) = v;
            }
            if (ch == 1) {
                for (int j = tid; j < qn * 2 * NC; j += blockDim.x) {
                    const int qq = j / (2 * NC), rr = (j / NC) % 2, c = j % NC;
                    const DescF& d = sh.desc[qq * 4 + 2 + rr];
                    const float* base = Gf + c * nsp;   // the on-site pair is its own exchange
                    const float* wgt = c == 0 ? d.wd : d.ws;
                    float v = 0.0f;
#pragma unroll
                    for (int k = 0; k < 4; ++k) v += wgt[k] * base[d.off[k]];
                    sh.onrow[(qq * 2 + rr) * NC + c] = v;
                }
            }
            __syncthreads();
            if (ch != 1) {
                if (site_on) {
                    const int r = my_r;
                    for (int q = my_g; q < qn; q += NG) {
                        float A[NC], B[NC];
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            A[c] = sh.rows[(q * 2) * rowp + c * nsp + r];
                            B[c] = sh.rows[(q * 2 + 1) * rowp + c * nsp + r];
                        }
                        if (ch == 0) su_product_acc<float, NC, -1>(A, B, racc); else su_product_acc<float, NC, 1>(A, B, racc);
                    }
                } else if (!site_reg) {
                    for (int r = tid; r < g.Ns; r += blockDim.x) {
                        float accl[NC], A[NC], B[NC];
#pragma unroll
                        for (int c = 0; c < NC; ++c) accl[c] = 0.0f;
                        for (int q = 0; q < qn; ++q) {
#pragma unroll
                            for (int c = 0; c < NC; ++c) {
                                A[c] = sh.rows[(q * 2) * rowp + c * nsp + r];
                                B[c] = sh.rows[(q * 2 + 1) * rowp + c * nsp + r];
                            }
                            if (ch == 0) su_product_acc<float, NC, -1>(A, B, accl); else su_product_acc<float, NC, 1>(A, B, accl);
                        }
#pragma unroll
                        for (int c = 0; c < NC; ++c) sh.acc[r * NC + c] += accl[c];
                    }
                }
            } else {
                if (tile_on) {
                    const int c = my_tile / (nsp4 * nsp4), ra = (my_tile / nsp4) % nsp4, rb = my_tile % nsp4;
                    for (int q = my_tg; q < qn; q += TG) {
                        const float4 av = *reinterpret_cast<const float4*>(sh.rows + (q * 2) * rowp + c * nsp + 4 * ra);
                        const float4 bv = *reinterpret_cast<const float4*>(sh.rows + (q * 2 + 1) * rowp + c * nsp + 4 * rb);
                        const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) a4[i][j] += ar[i] * br[j];
                    }
                } else if (DENSE && !tile_reg) {
                    for (int tl = tid; tl < ntile; tl += blockDim.x) {
                        const int c = tl / (nsp4 * nsp4), ra = (tl / nsp4) % nsp4, rb = tl % nsp4;
                        float t4[4][4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) t4[i][j] = 0.0f;
                        for (int q = 0; q < qn; ++q) {
                            const float4 av = *reinterpret_cast<const float4*>(sh.rows + (q * 2) * rowp + c * nsp + 4 * ra);
                            const float4 bv = *reinterpret_cast<const float4*>(sh.rows + (q * 2 + 1) * rowp + c * nsp + 4 * rb);
                            const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                            for (int i = 0; i < 4; ++i)
#pragma unroll
                                for (int j = 0; j < 4; ++j) t4[i][j] += ar[i] * br[j];
                        }
                        float* cp = sh.cacc + c * nsp * nsp + (4 * ra) * nsp + 4 * rb;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            float4 cv = *reinterpret_cast<float4*>(cp + i * nsp);
                            cv.x += t4[i][0]; cv.y += t4[i][1]; cv.z += t4[i][2]; cv.w += t4[i][3];
                            *reinterpret_cast<float4*>(cp + i * nsp) = cv;
                        }
                    }
                } else if (!DENSE) {
                    for (int o = tid; o < tb.nprod; o += blockDim.x) {
                        const int2 pr = tb.prodp[o];
                        float a = 0.0f;
                        for (int q = 0; q < qn; ++q) a += sh.rows[(q * 2) * rowp + pr.x] * sh.rows[(q * 2 + 1) * rowp + pr.y];
                        sh.cacc[o] += a;
                    }
                }
                // on-site terms
                if (site_on) {
                    const int r = my_r;
                    const int pon = tb.onsite_perm[r];
                    for (int q = my_g; q < qn; q += NG) {
                        float A[NC], B[NC], Cp[NC], D[NC];
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            A[c] = sh.rows[(q * 2) * rowp + c * nsp + r];
                            B[c] = sh.rows[(q * 2 + 1) * rowp + c * nsp + r];
                            Cp[c] = sh.onrow[(q * 2) * NC + perm_of(pon, c)];
                            D[c] = sh.onrow[(q * 2 + 1) * NC + c];
                        }
#pragma unroll
                        for (int c = 0; c < NC; ++c)
                            racc[c] = fmadd(A[c], onsite_factor<float, NC>(Cp, c), fmadd(onsite_factor<float, NC>(D, c), B[c], racc[c]));
                    }
                } else if (!site_reg) {
                    for (int r = tid; r < g.Ns; r += blockDim.x) {
                        const int pon = tb.onsite_perm[r];
                        float accl[NC];
#pragma unroll
                        for (int c = 0; c < NC; ++c) accl[c] = 0.0f;
                        for (int q = 0; q < qn; ++q) {
                            float A[NC], B[NC], Cp[NC], D[NC];
#pragma unroll
                            for (int c = 0; c < NC; ++c) {
                                A[c] = sh.rows[(q * 2) * rowp + c * nsp + r];
                                B[c] = sh.rows[(q * 2 + 1) * rowp + c * nsp + r];
                                Cp[c] = sh.onrow[(q * 2) * NC + perm_of(pon, c)];
                                D[c] = sh.onrow[(q * 2 + 1) * NC + c];
                            }
#pragma unroll
                            for (int c = 0; c < NC; ++c)
                                accl[c] = fmadd(A[c], onsite_factor<float, NC>(Cp, c), fmadd(onsite_factor<float, NC>(D, c), B[c], accl[c]));
                        }
#pragma unroll
                        for (int c = 0; c < NC; ++c) sh.acc[r * NC + c] += accl[c];
                    }
                }
            }
        }
        // end of the channel: combine the register partials of the node groups in a fixed order
        // (scratch: the row buffer, free once the channel's last node block is done)
        __syncthreads();
        float* scr = sh.rows;
        if (site_on) {
#pragma unroll
            for (int c = 0; c < NC; ++c) scr[(my_g * NC + c) * g.Ns + my_r] = racc[c];
        }
        float* scr2 = sh.rows + (site_reg ? NG * g.Ns * NC : 0);
        if (ch == 1 && tile_on) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) scr2[(my_tg * 16 + i * 4 + j) * ntile + my_tile] = a4[i][j];
        }
        __syncthreads();
        if (site_reg)
            for (int o = tid; o < g.Ns * NC; o += blockDim.x) {
                const int r = o / NC, c = o % NC;
                float a = 0.0f;
                for (int k = 0; k < NG; ++k) a += scr[(k * NC + c) * g.Ns + r];
                sh.acc[o] += a;
            }
        if (ch == 1 && tile_reg)
            for (int e = tid; e < ntile * 16; e += blockDim.x) {
                const int tl = e % ntile, ij = e / ntile;
                float a = 0.0f;
                for (int k = 0; k < TG; ++k) a += scr2[(k * 16 + ij) * ntile + tl];
                const int c = tl / (nsp4 * nsp4), ra = (tl / nsp4) % nsp4, rb = tl % nsp4;
                sh.cacc[c * nsp * nsp + (4 * ra + (ij >> 2)) * nsp + 4 * rb + (ij & 3)] += a;
            }
    }
    __syncthreads();
    const int* gidx = DENSE ? tb.dgath_idx : tb.gath_idx;
    for (int o = tid; o < g.Ns * NC; o += blockDim.x) {
        const int r = o / NC, c = o % NC;
        float a = 0.0f;
        for (int k = tb.gath_off[o]; k < tb.gath_off[o + 1]; ++k) a += sh.cacc[gidx[k]];
        dG[((size_t)(p * g.N + ti) * NC + c) * g.Ns + r] = (double)sh.acc[o] - 2.0 * (double)a;
    }
}

template <int NC, bool DENSE>
__global__ void __launch_bounds__(kThreads) k_gamma_rhs_f32(Geo g, Tabs tb, const float* __restrict__ Gf,
                                                            const float* __restrict__ Gs, const float* __restrict__ nx,
                                                            const float* __restrict__ nW, const int* __restrict__ ncount,
                                                            double* __restrict__ dG, int p0) {
    extern __shared__ __align__(16) unsigned char smem[];
    gamma_rhs_f32_triple<NC, DENSE>(g, tb, Gf, Gs, nx, nW, ncount, dG, p0 + (int)(blockIdx.x / g.N), blockIdx.x % g.N, smem, kQF);
}

// The SU2 kernel with the lattice sum on the tensor cores, persistent: each CTA allocates its
// TMEM accumulator and MMA barrier once and takes the stored triples blockIdx.x,
// blockIdx.x + gridDim.x, ...; the grid is sized so that the CTAs resident on an SM never ask
// for more than its 512 TMEM columns.  `fail` is set if an MMA completion wait gives up (the
// outputs of that triple are then NaN, so the flow's finiteness check reports it).
static_assert(kThreads == 128, "the TMEM read-back maps the four warps onto the four lane quarters");
__global__ void __launch_bounds__(kThreads) k_gamma_rhs_f32_tc(Geo g, Tabs tb, const float* __restrict__ Gf,
                                                               const float* __restrict__ Gs, const float* __restrict__ nx,
                                                               const float* __restrict__ nW, const int* __restrict__ ncount,
                                                               double* __restrict__ dG, int* __restrict__ fail, long u0, long u1) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    const uint32_t ncols = (uint32_t)tc_shape(g.nsp).ncols;
    if (threadIdx.x == 0) { tc::mbar_init(&mbar); failed = 0; }
    if (threadIdx.x < 32) tc::tmem_alloc(&tmem_slot, ncols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    TcCta tcs{tmem_slot, &mbar, 0u, &failed};
    for (long tr = u0 + blockIdx.x; tr < u1; tr += gridDim.x) {   // triples (units) u0 .. u1 - 1
        const int p = (int)(tr / g.N), ti = (int)(tr % g.N);
        gamma_rhs_f32_triple<2, true, true>(g, tb, Gf, Gs, nx, nW, ncount, dG, p, ti, smem, kQF, &tcs);
        __syncthreads();
        if (failed) {
            for (int o = threadIdx.x; o < g.Ns * 2; o += blockDim.x)
                dG[((size_t)(p * g.N + ti) * 2 + o % 2) * g.Ns + o / 2] = __longlong_as_double(0x7ff8000000000000LL);
            if (threadIdx.x == 0) atomicOr(fail, 1);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(tcs.tmem, ncols);
}

#include "su2f.cuh"

// FP32 shadow of the state in the padded layout, and (with_swap) the exchanged copy in which
// entry (c, r) holds the stored value of the pair (rep_r, ref): component perm(c) of site
// swap_r[r].  Padding sites are zero.
__global__ void k_shadow(Geo g, Tabs tb, const double* __restrict__ G, float* __restrict__ Gf, int with_swap) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= g.nentp) return;
    const int rowp = g.nc * g.nsp;
    const long pt = i / rowp;
    const int rem = (int)(i % rowp);
    const int c = rem / g.nsp, r = rem % g.nsp;
    const double* src = G + pt * g.nc * g.Ns;
    float v = 0.0f, vs = 0.0f;
    if (r < g.Ns) {
        v = (float)src[c * g.Ns + r];
        if (with_swap) vs = (float)src[perm_of(tb.swap_perm[r], c) * g.Ns + tb.swap_r[r]];
    }
    Gf[i] = v;
    if (with_swap) Gf[g.nentp + i] = vs;
}

template <typename T>
__global__ void k_fill_init(Geo g, const T* __restrict__ init /* Ns * nc */, T* __restrict__ G) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= g.nent) return;
    int r = (int)(i % g.Ns);
    int c = (int)((i / g.Ns) % g.nc);
    G[i] = init[r * g.nc + c];
}


// y <- y + a f, flagging non-finite results.
__global__ void k_axpy(long n, double* __restrict__ y, const double* __restrict__ f, double a, int* __restrict__ flag) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = y[i] + a * f[i];
    if (!isfinite(v)) atomicOr(flag, 1);
    y[i] = v;
}

struct KPtrs { const double* k[7]; };

// Dormand-Prince stage state: out = y0 + h sum_{r < s} a_r k_r.
__global__ void k_rk_stage(long n, const double* __restrict__ y0, KPtrs kp, int s, double a0, double a1, double a2,
                           double a3, double a4, double a5, double h, double* __restrict__ out) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a[6] = {a0, a1, a2, a3, a4, a5};
    double acc = 0.0;
    for (int r = 0; r < s; ++r) acc += a[r] * kp.k[r][i];
    out[i] = y0[i] + h * acc;
}

// Fifth-order solution; the block-wise maxima of |h (y5 - y4)| and of max(|y0|, |y_new|) are
// combined with atomicMax on their (non-negative) bit patterns, which is exact and
// order-independent: errbits[0] = max error, errbits[1] = max magnitude.
__global__ void k_rk_final(long n, const double* __restrict__ y0, KPtrs kp, double h, double* __restrict__ out,
                           unsigned long long* __restrict__ errbits, int* __restrict__ flag) {
    const double b5[7] = {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0.0};
    const double b4[7] = {5179.0 / 57600, 0.0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    double e = 0.0, y = 0.0;
    if (i < n) {
        double y5 = 0.0, y4 = 0.0;
        for (int r = 0; r < 7; ++r) { double kv = kp.k[r][i]; y5 += b5[r] * kv; y4 += b4[r] * kv; }
        double yn = y0[i] + h * y5;
        e = fabs(h * (y5 - y4));
        y = fmax(fabs(y0[i]), fabs(yn));
        if (!isfinite(yn) || !isfinite(e)) atomicOr(flag, 1);
        out[i] = yn;
    }
    for (int o = 16; o > 0; o >>= 1) {
        e = fmax(e, __shfl_down_sync(0xffffffffu, e, o));
        y = fmax(y, __shfl_down_sync(0xffffffffu, y, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (e > 0.0) atomicMax(errbits, (unsigned long long)__double_as_longlong(e));
        if (y > 0.0) atomicMax(errbits + 1, (unsigned long long)__double_as_longlong(y));
    }
}

// Correlations chi^{cc}_{b j} (Eq. frg:correlation), one block per (b, j): bubble (local)
// plus the product-trapezoid vertex term with the exact G^2 weights of each segment.
template <typename T, int NC>
__global__ void k_chi(Geo g, Tabs tb, const double* __restrict__ w, const T* __restrict__ gam,
                      const T* __restrict__ G, double lam, const int2* __restrict__ cmap,
                      const int* __restrict__ onsite, int ntot, T* __restrict__ chi) {
    __shared__ double y[kMaxFreq + 1];
    __shared__ __align__(16) unsigned char wn_raw[sizeof(T) * (kMaxFreq + 1)];
    __shared__ double red[NC * 32 * (sizeof(T) / sizeof(double))];
    __shared__ int Ksh;
    T* Wn = reinterpret_cast<T*>(wn_raw);
    const int pidx = blockIdx.x;      // b * ntot + j
    const int b = pidx / ntot;
    const int on = onsite[pidx];
    const int2 pm = cmap[pidx];
    const int2 pon = cmap[b * ntot + 0];  // the first site of each list is (0, b) itself
    const int N = g.N;
    if (threadIdx.x == 0) {
        int K = 0;
        y[K++] = lam;
        for (int i = 0; i < N; ++i) if (w[i] > lam) y[K++] = w[i];
        for (int k = 0; k < K; ++k) Wn[k] = T(0.0);
        for (int k = 0; k + 1 < K; ++k) {
            const T ya = y[k] + interp_odd(w, tb.invh, N, gam, y[k]);
            const T yb = y[k + 1] + interp_odd(w, tb.invh, N, gam, y[k + 1]);
            const T seg = (y[k + 1] - y[k]) / (ya * yb);
            Wn[k] += 0.5 * seg;
            Wn[k + 1] += 0.5 * seg;
        }
        Wn[K - 1] += 1.0 / (y[K - 1] + interp_odd(w, tb.invh, N, gam, y[K - 1]));
        Ksh = K;
    }
    __syncthreads();
    const int K = Ksh, M = 2 * K;
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = T(0.0);
    for (int idx = threadIdx.x; idx < M * M; idx += blockDim.x) {
        const int pi = idx / M, qi = idx % M;
        const double xp = pi < K ? y[pi] : -y[pi - K];
        const double xq = qi < K ? y[qi] : -y[qi - K];
        const T wpq = Wn[pi % K] * Wn[qi % K];
        Desc<double> d;
        make_desc(xp + xq, 0.0, xp - xq, 1, 0, tb, g, d);
        T v[NC], e[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = row_value(G, d, tb, g, pm.x, perm_of(pm.y, c));
        if (on) {
            make_desc(xp + xq, xq - xp, 0.0, 2, 0, tb, g, d);
#pragma unroll
            for (int c = 0; c < NC; ++c) e[c] = row_value(G, d, tb, g, pon.x, perm_of(pon.y, c));
        }
#pragma unroll
        for (int mu = 0; mu < NC; ++mu) {
            T F = 4.0 * v[mu];
            if (on) {
                T x;
                if (NC == 2) x = mu == 0 ? T(2.0 * (e[0] + 3.0 * e[1])) : T(2.0 * (e[0] - e[1]));
                else {
                    x = T(0.0);
                    for (int k = 0; k < 4; ++k) x += (mu == 0 || k == 0 || k == mu) ? T(2.0 * e[k]) : T(-2.0 * e[k]);
                }
                F -= x;
            }
            acc[mu] += wpq * F;
        }
    }
    block_sum<T, NC>(acc, red);
    if (threadIdx.x == 0) {
        T bub = T(0.0);
        for (int k = 0; k < K; ++k) bub += Wn[k];
        bub = bub / (2.0 * kPi);
        for (int mu = 0; mu < NC; ++mu)
            chi[(size_t)pidx * NC + mu] = (on ? bub : T(0.0)) - acc[mu] / (16.0 * kPi * kPi);
    }
}

// chi(k) = (1/N_b) sum_{b, j} cos(k (r_b - r_j)) sum_{mu = x,y,z} chi^{mu mu}_{b j}.
template <typename T>
__global__ void k_chi_k(int nk, const double* __restrict__ kp, const T* __restrict__ chi,
                        const double* __restrict__ dr, int npairs, int nb, int nc, T* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nk) return;
    const double kx = kp[3 * i], ky = kp[3 * i + 1], kz = kp[3 * i + 2];
    T acc = T(0.0);
    for (int p = 0; p < npairs; ++p) {
        const T sp = nc == 2 ? T(3.0 * chi[(size_t)p * 2 + 1]) : T(chi[(size_t)p * 4 + 1] + chi[(size_t)p * 4 + 2] + chi[(size_t)p * 4 + 3]);
        acc += cos(kx * dr[3 * p] + ky * dr[3 * p + 1] + kz * dr[3 * p + 2]) * sp;
    }
    out[i] = acc / (double)nb;
}

}  // namespace

#include "adjoint.cuh"
#include "tri.cuh"
#include "tri_adj.cuh"

// ----------------------------------------------------------------------------- objects

template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t count) {
        if (p) { cudaFree(p); p = nullptr; }
        n = count;
        if (count == 0) return cudaSuccess;
        return cudaMalloc((void**)&p, sizeof(T) * count);
    }
    cudaError_t upload(const T* host, size_t count, cudaStream_t st) {
        cudaError_t e = alloc(count);
        if (e != cudaSuccess || count == 0) return e;
        return cudaMemcpyAsync(p, host, sizeof(T) * count, cudaMemcpyHostToDevice, st);
    }
};

struct sr_flow {
    const sr_lattice* lat = nullptr;
    Geo g{};
    sr_precision prec = SR_FP64;
    cudaStream_t stream = nullptr;
    int device = -1;                 // CUDA device current when the flow was created
    double lambda = 0.0;
    std::vector<double> mesh;
    int ntan = 0;   // tangent directions (0: plain flow; kTan: the state holds Dual<kTan> values)
    int ts = 1;     // doubles per state scalar

    DevBuf<double> w, gam, G, dgam, dG;
    DevBuf<float> Gf;
    DevBuf<double> nx, nW;
    DevBuf<float> nWf, nxf;
    DevBuf<int> ncount;
    DevBuf<int> swap_r, swap_perm, onsite_perm, mult, gath_off, gath_idx;
    DevBuf<int2> prod;
    DevBuf<double> invh;
    DevBuf<float> wf, invhf;
    DevBuf<int2> prodp;
    DevBuf<int> dgath_idx;
    bool has_swap = false, dense = false;
    bool use_tc = false;          // FP32-mixed SU2: lattice sum on the tensor cores
    size_t smem_su2f = 0;         // FP32-mixed SU2 kernel (k_gamma_rhs_su2f): dynamic shared memory,
    int su2f_qb = 0;              // its integration nodes per block (0: the kernel is not used)
    size_t smem_tc = 0;           // dynamic shared memory of the tensor-core kernel
    int tc_grid = 0;              // its persistent grid (SMs x resident CTAs)
    int tc_occ_api = 0;           // the runtime's occupancy figure for it (reported only)
    DevBuf<int> tcfail;           // set by the tensor-core kernel when an MMA wait gives up
    int nprod = 0;
    DevBuf<double> init;
    DevBuf<int2> chi_map;
    DevBuf<int> chi_onsite;
    DevBuf<double> chi_dr, chi, kbuf, chik;
    DevBuf<int> flag;
    DevBuf<unsigned long long> errbits;
    // Dormand-Prince work space (allocated on first use)
    DevBuf<double> y0g, y0G, stg, stG;
    DevBuf<double> kg[7], kG[7];
    // launch timing (measurement only): event pairs per kernel id
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[3];
    double last_err = 0.0, h_next = 0.0;
    double err_prev = 1e-4;      // error norm of the last accepted adaptive step (controller memory)
    bool fsal = false;           // kg[6] / kG[6] hold the right-hand side of the current state
    long step_limit = 1000000;   // attempted steps per sr_flow_step call
    long n_rhs = 0, n_accept = 0, n_reject = 0;
    size_t smem_rhs = 0;
    // lattice-sum tables on the host (the adjoint inverts them on first use)
    std::vector<int2> h_prod;
    std::vector<int> h_goff, h_gidx;
    // adjoint work space (allocated on first use)
    bool adj_ready = false;
    size_t smem_adj = 0;
    DevBuf<int> pinv_off, pinv_out, ainv_off, ainv_idx, binv_off, binv_idx;
    DevBuf<double> ntw, Wbar, dgbar, tg, tG, chibar, kbar;
    // TRI core tables (nc = 16)
    DevBuf<int> swap_map16, onsite_map16, tlat_item_off, tlat_off, chi_r16, chi_m16;
    DevBuf<int2> tlat_ent;
    DevBuf<uint4> tlat_rec;
    DevBuf<int4> tlat_items;
    int tlat_n_items = 0;

    Tabs tabs() const {
        Tabs t;
        t.swap_r = swap_r.p; t.swap_perm = swap_perm.p; t.onsite_perm = onsite_perm.p; t.mult = mult.p;
        t.prod = prod.p; t.gath_off = gath_off.p; t.gath_idx = gath_idx.p; t.nprod = nprod; t.invh = invh.p;
        t.w = w.p; t.wf = wf.p; t.invhf = invhf.p; t.prodp = prodp.p; t.dgath_idx = dgath_idx.p;
        return t;
    }
    TabsT tabs_tri() const {
        TabsT t;
        t.swap_map = swap_map16.p; t.onsite_map = onsite_map16.p; t.lat_rec = tlat_rec.p; t.lat_items = tlat_items.p;
        t.lat_item_off = tlat_item_off.p; t.n_items = tlat_n_items; t.lat_off = tlat_off.p; t.lat_ent = tlat_ent.p;
        return t;
    }
};

// The dynamic shared-memory limit is a property of the kernel, shared by every flow: raise
// it to the largest size any flow has asked for, never lower it.
static std::mutex g_smem_mu;
static std::map<std::pair<int, const void*>, int> g_smem_max;

static cudaError_t ensure_smem(const void* kernel, size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_smem_mu);
    int& cur = g_smem_max[{dev, kernel}];
    if ((int)bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = (int)bytes;
    return e;
}

static int pack_perm(const sr::Perm& p) { return p[0] | (p[1] << 2) | (p[2] << 4) | (p[3] << 6); }

static size_t rhs_smem_bytes(const Geo& g, int nprod, size_t tsz) {
    const size_t dsz = sizeof(Desc<double>);
    auto rnd = [](size_t b) { return (b + 15) & ~size_t(15); };
    return rnd(dsz * kQC * 4) + rnd(tsz * g.Ns * g.nc) + rnd(tsz * nprod) + rnd(tsz * kQC * 2 * g.Ns * g.nc) +
           rnd(tsz * kQC * 2 * g.nc) + rnd(tsz * kQC);
}

static sr_status prof_begin(sr_flow* f, int id, cudaEvent_t* b) {
    if (!f->profiling) return SR_OK;
    CK(cudaEventCreate(b));
    CK(cudaEventRecord(*b, f->stream));
    (void)id;
    return SR_OK;
}
static sr_status prof_end(sr_flow* f, int id, cudaEvent_t b) {
    if (!f->profiling) return SR_OK;
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    CK(cudaEventRecord(e, f->stream));
    f->ev[id].push_back({b, e});
    return SR_OK;
}

// Right-hand side at cutoff lam for the state (gam_s, G_s [, Gf_s]) into (dgam_o, dG_o).
static sr_status run_rhs(sr_flow* f, double lam, const double* gam_s, const double* G_s, const float* Gf_s,
                         double* dgam_o, double* dG_o, int pb = 0, int pe = -1) {
    const Geo& g = f->g;
    Tabs tb = f->tabs();
    cudaEvent_t e0 = nullptr;
    if (pe < 0) pe = g.npair;   // stored (s, u) pairs pb .. pe - 1 (all by default)
    const int blocks = (pe - pb) * g.N;
    if (f->ntan) {
        // tangent-linear flow: the same kernels on dual numbers
        const DualT* gs = reinterpret_cast<const DualT*>(gam_s);
        const DualT* Gd = reinterpret_cast<const DualT*>(G_s);
        DualT* dgo = reinterpret_cast<DualT*>(dgam_o);
        DualT* dGo = reinterpret_cast<DualT*>(dG_o);
        DualT* nW = reinterpret_cast<DualT*>(f->nW.p);
        if (sr_status s = prof_begin(f, 0, &e0)) return s;
        if (g.nc == 16)
            k_sigma_rhs_tri<DualT><<<g.N, 64, 0, f->stream>>>(g, tb, f->tabs_tri(), f->w.p, gs, Gd, lam, dgo);
        else
            k_sigma_rhs<DualT><<<g.N, 64, 0, f->stream>>>(g, tb, f->w.p, gs, Gd, lam, dgo);
        if (sr_status s = prof_end(f, 0, e0)) return s;
        if (sr_status s = prof_begin(f, 1, &e0)) return s;
        k_channel_nodes<DualT><<<3 * g.N, 128, 0, f->stream>>>(g, f->w.p, f->invh.p, gs, dgo, lam, f->nx.p, nW, nullptr, f->ncount.p,
                                                              nullptr);
        if (sr_status s = prof_end(f, 1, e0)) return s;
        if (sr_status s = prof_begin(f, 2, &e0)) return s;
        if (g.nc == 16)
            k_gamma_rhs_tri<DualT><<<blocks, kThreads, f->smem_rhs, f->stream>>>(g, tb, f->tabs_tri(), f->w.p, Gd, f->nx.p, nW,
                                                                                   f->ncount.p, dGo, pb);
        else if (g.nc == 2)
            k_gamma_rhs<DualT, 2><<<blocks, kThreads, f->smem_rhs, f->stream>>>(g, tb, f->w.p, Gd, f->nx.p, nW, f->ncount.p, dGo, pb);
        else
            k_gamma_rhs<DualT, 4><<<blocks, kThreads, f->smem_rhs, f->stream>>>(g, tb, f->w.p, Gd, f->nx.p, nW, f->ncount.p, dGo, pb);
        if (sr_status s = prof_end(f, 2, e0)) return s;
        CK(cudaGetLastError());
        f->n_rhs++;
        return SR_OK;
    }
    if (g.nc == 16) {
        // TRI core: FP64 state and lookups; rows and products in FP64 or FP32
        const TabsT tt = f->tabs_tri();
        if (sr_status s = prof_begin(f, 0, &e0)) return s;
        k_sigma_rhs_tri<<<g.N, 64, 0, f->stream>>>(g, tb, tt, f->w.p, gam_s, G_s, lam, dgam_o);
        if (sr_status s = prof_end(f, 0, e0)) return s;
        if (sr_status s = prof_begin(f, 1, &e0)) return s;
        k_channel_nodes<double><<<3 * g.N, 128, 0, f->stream>>>(g, f->w.p, f->invh.p, gam_s, dgam_o, lam, f->nx.p, f->nW.p, f->nWf.p,
                                                               f->ncount.p, nullptr);
        if (sr_status s = prof_end(f, 1, e0)) return s;
        if (sr_status s = prof_begin(f, 2, &e0)) return s;
        if (f->prec == SR_FP64)
            k_gamma_rhs_tri<double><<<blocks, kThreads, f->smem_rhs, f->stream>>>(g, tb, tt, f->w.p, G_s, f->nx.p, f->nW.p, f->ncount.p, dG_o, pb);
        else
            k_gamma_rhs_tri<float><<<blocks, kThreads, f->smem_rhs, f->stream>>>(g, tb, tt, f->w.p, Gf_s, f->nx.p, f->nW.p, f->ncount.p, dG_o, pb);
        if (sr_status s = prof_end(f, 2, e0)) return s;
        CK(cudaGetLastError());
        f->n_rhs++;
        return SR_OK;
    }
    if (sr_status s = prof_begin(f, 0, &e0)) return s;
    k_sigma_rhs<double><<<g.N, 64, 0, f->stream>>>(g, tb, f->w.p, gam_s, G_s, lam, dgam_o);
    if (sr_status s = prof_end(f, 0, e0)) return s;
    if (sr_status s = prof_begin(f, 1, &e0)) return s;
    k_channel_nodes<double><<<3 * g.N, 128, 0, f->stream>>>(g, f->w.p, f->invh.p, gam_s, dgam_o, lam, f->nx.p, f->nW.p, f->nWf.p,
                                                           f->ncount.p, f->prec == SR_FP32_MIXED ? f->nxf.p : nullptr);
    if (sr_status s = prof_end(f, 1, e0)) return s;
    if (sr_status s = prof_begin(f, 2, &e0)) return s;
    if (f->prec == SR_FP64) {
        if (g.nc == 2)
            k_gamma_rhs<double, 2><<<blocks, kThreads, f->smem_rhs, f->stream>>>(g, tb, f->w.p, G_s, f->nx.p, f->nW.p, f->ncount.p, dG_o, pb);
        else
            k_gamma_rhs<double, 4><<<blocks, kThreads, f->smem_rhs, f->stream>>>(g, tb, f->w.p, G_s, f->nx.p, f->nW.p, f->ncount.p, dG_o, pb);
    } else {
        const float* Gs = f->has_swap ? Gf_s + g.nentp : Gf_s;
        if (g.nc == 2 && f->dense && f->use_tc)
            k_gamma_rhs_f32_tc<<<std::min(blocks, f->tc_grid), kThreads, f->smem_tc, f->stream>>>(g, tb, Gf_s, Gs, f->nxf.p, f->nWf.p, f->ncount.p, dG_o,
                                                                            f->tcfail.p, (long)pb * g.N, (long)pe * g.N);
        else if (g.nc == 2 && f->dense && f->su2f_qb > 0 && su2f::cache_for(g.nsp))
            k_gamma_rhs_su2f<true><<<blocks, su2f::threads_for(g.nsp), f->smem_su2f, f->stream>>>(
                g, tb, Gf_s, f->has_swap ? (int)g.nentp : 0, f->nxf.p, f->nWf.p, f->ncount.p, dG_o, f->su2f_qb, pb);
        else if (g.nc == 2 && f->dense && f->su2f_qb > 0)
            k_gamma_rhs_su2f<false><<<blocks, su2f::threads_for(g.nsp), f->smem_su2f, f->stream>>>(
                g, tb, Gf_s, f->has_swap ? (int)g.nentp : 0, f->nxf.p, f->nWf.p, f->ncount.p, dG_o, f->su2f_qb, pb);
        else if (g.nc == 2 && f->dense)
            k_gamma_rhs_f32<2, true><<<blocks, kThreads, f->smem_rhs, f->stream>>>(g, tb, Gf_s, Gs, f->nxf.p, f->nWf.p, f->ncount.p, dG_o, pb);
        else if (g.nc == 2)
            k_gamma_rhs_f32<2, false><<<blocks, kThreads, f->smem_rhs, f->stream>>>(g, tb, Gf_s, Gs, f->nxf.p, f->nWf.p, f->ncount.p, dG_o, pb);
        else
            k_gamma_rhs_f32<4, false><<<blocks, kThreads, f->smem_rhs, f->stream>>>(g, tb, Gf_s, Gs, f->nxf.p, f->nWf.p, f->ncount.p, dG_o, pb);
    }
    if (sr_status s = prof_end(f, 2, e0)) return s;
    CK(cudaGetLastError());
    f->n_rhs++;
    return SR_OK;
}

static sr_status refresh_shadow(sr_flow* f, const double* G_s, float* Gf_s) {
    if (f->prec != SR_FP32_MIXED) return SR_OK;
    if (f->g.nc == 16) {
        const long n = f->g.nent;
        k_shadow_tri<<<(unsigned)((n + 255) / 256), 256, 0, f->stream>>>(n, G_s, Gf_s);
        CK(cudaGetLastError());
        return SR_OK;
    }
    long n = f->g.nentp;
    k_shadow<<<(unsigned)((n + 255) / 256), 256, 0, f->stream>>>(f->g, f->tabs(), G_s, Gf_s, f->has_swap ? 1 : 0);
    CK(cudaGetLastError());
    return SR_OK;
}

// ----------------------------------------------------------------------------- ABI: lattice

extern "C" sr_status sr_lattice_create(const sr_lattice_desc* desc, sr_lattice** out) {
    if (!desc || !out) return fail(SR_EINVAL, "null argument");
    *out = nullptr;
    if (desc->n_basis <= 0 || !desc->basis_xyz) return fail(SR_EINVAL, "n_basis must be positive with basis_xyz given");
    if (desc->n_bonds <= 0 || !desc->bonds) return fail(SR_EINVAL, "at least one bond is required");
    if (desc->n_couplings < 0 || (desc->n_couplings > 0 && !desc->couplings)) return fail(SR_EINVAL, "bad couplings");
    if (desc->range_L < 0 || desc->range_L > 64) return fail(SR_EINVAL, "range_L must be in [0, 64]");
    if (desc->backend != SR_SU2 && desc->backend != SR_XYZ && desc->backend != SR_TRI) return fail(SR_EINVAL, "unknown backend");
    std::unique_ptr<sr_lattice> lat(new (std::nothrow) sr_lattice());
    if (!lat) return fail(SR_ENOMEM, "out of host memory");
    std::string msg;
    sr_status st;
    try {
        st = sr::build_lattice(desc, lat.get(), &msg);
    } catch (const std::bad_alloc&) {
        return fail(SR_ENOMEM, "out of host memory");
    } catch (...) {
        return fail(SR_EINVAL, "lattice construction failed");
    }
    if (st != SR_OK) return fail(st, "%s", msg.c_str());
    *out = lat.release();
    return SR_OK;
}

extern "C" sr_status sr_lattice_info(const sr_lattice* lat, int* N_s, int* N_tot, int* N_basis, long* P) {
    if (!lat) return fail(SR_EINVAL, "null lattice");
    if (N_s) *N_s = lat->Ns;
    if (N_tot) *N_tot = lat->Ntot;
    if (N_basis) *N_basis = lat->nb;
    if (P) *P = (long)lat->rpa.size();
    return SR_OK;
}

extern "C" sr_status sr_lattice_representatives(const sr_lattice* lat, int* rep) {
    if (!lat || !rep) return fail(SR_EINVAL, "null argument");
    for (int r = 0; r < lat->Ns; ++r) {
        const sr::SiteKey& s = lat->sites[lat->rep[r]];
        rep[4 * r] = s.n[0]; rep[4 * r + 1] = s.n[1]; rep[4 * r + 2] = s.n[2]; rep[4 * r + 3] = s.b;
    }
    return SR_OK;
}

extern "C" sr_status sr_lattice_map_pair(const sr_lattice* lat, const int* i1, const int* i2, int* r, int* perm) {
    if (!lat || !i1 || !i2 || !r) return fail(SR_EINVAL, "null argument");
    if (i1[3] < 0 || i1[3] >= lat->nb || i2[3] < 0 || i2[3] >= lat->nb) return fail(SR_EINVAL, "basis index out of range");
    sr::SiteKey a{{i1[0], i1[1], i1[2]}, i1[3]}, b{{i2[0], i2[1], i2[2]}, i2[3]};
    sr::PairMap pm = lat->map_pair(a, b);
    *r = pm.r;
    if (perm) for (int c = 0; c < 4; ++c) perm[c] = lat->backend == SR_SU2 ? c : pm.perm[c];
    return SR_OK;
}

extern "C" sr_status sr_lattice_map_pair_components(const sr_lattice* lat, const int* i1, const int* i2, int* r, int* comp,
                                                    int* sign) {
    if (!lat || !i1 || !i2 || !r || !comp || !sign) return fail(SR_EINVAL, "null argument");
    if (i1[3] < 0 || i1[3] >= lat->nb || i2[3] < 0 || i2[3] >= lat->nb) return fail(SR_EINVAL, "basis index out of range");
    sr::SiteKey a{{i1[0], i1[1], i1[2]}, i1[3]}, b{{i2[0], i2[1], i2[2]}, i2[3]};
    if (lat->nc == 16) {
        const sr::PairMap16 pm = lat->map_pair16(a, b);
        *r = pm.r;
        for (int c = 0; c < 16; ++c) { comp[c] = pm.m[c] & 15; sign[c] = (pm.m[c] & 16) ? -1 : 1; }
        return SR_OK;
    }
    const sr::PairMap pm = lat->map_pair(a, b);
    *r = pm.r;
    for (int c = 0; c < lat->nc; ++c) { comp[c] = lat->backend == SR_SU2 ? c : pm.perm[c]; sign[c] = 1; }
    return SR_OK;
}

extern "C" sr_status sr_lattice_destroy(sr_lattice* lat) {
    delete lat;
    return SR_OK;
}

extern "C" sr_status sr_frequency_mesh_exponential(int n, double wmin, double wmax, double* out) {
    if (n < 2 || !(wmin > 0.0) || !(wmax > wmin) || !out) return fail(SR_EINVAL, "need n >= 2 and 0 < w_min < w_max");
    for (int i = 0; i < n; ++i) out[i] = wmin * std::pow(wmax / wmin, (double)i / (double)(n - 1));
    return SR_OK;
}

// ----------------------------------------------------------------------------- ABI: flow

static sr_status flow_create(const sr_lattice* lat, int n_freq, const double* freq_pos, double lambda_init,
                             sr_precision precision, void* cuda_stream, int npar, const double* dM, sr_flow** out) {
    if (!lat || !freq_pos || !out) return fail(SR_EINVAL, "null argument");
    *out = nullptr;
    if (n_freq < 2 || n_freq > kMaxFreq) return fail(SR_EINVAL, "n_freq must be in [2, %d]", kMaxFreq);
    for (int i = 0; i < n_freq; ++i) {
        if (!(freq_pos[i] > 0.0) || !std::isfinite(freq_pos[i])) return fail(SR_EINVAL, "frequencies must be positive and finite");
        if (i > 0 && !(freq_pos[i] > freq_pos[i - 1])) return fail(SR_EINVAL, "frequencies must be strictly ascending");
    }
    if (!(lambda_init > 0.0) || !std::isfinite(lambda_init)) return fail(SR_EINVAL, "lambda_init must be positive");
    if (precision != SR_FP64 && precision != SR_FP32_MIXED) return fail(SR_EINVAL, "unknown precision");
    std::unique_ptr<sr_flow> f(new (std::nothrow) sr_flow());
    if (!f) return fail(SR_ENOMEM, "out of host memory");
    f->lat = lat;
    f->prec = precision;
    f->stream = (cudaStream_t)cuda_stream;
    CK(cudaGetDevice(&f->device));
    f->ntan = npar > 0 ? kTan : 0;
    f->ts = 1 + f->ntan;
    const int ts = f->ts;
    std::vector<double> init_host = lat->init_gamma;
    if (npar > 0) {
        std::vector<double> dinit;
        std::string msg;
        if (sr_status s = sr::tangent_init(lat, npar, dM, &dinit, &msg)) return fail(s, "%s", msg.c_str());
        init_host.assign(lat->init_gamma.size() * ts, 0.0);
        for (size_t e = 0; e < lat->init_gamma.size(); ++e) {
            init_host[e * ts] = lat->init_gamma[e];
            for (int p = 0; p < npar; ++p) init_host[e * ts + 1 + p] = dinit[e * npar + p];
        }
    }
    f->lambda = lambda_init;
    f->mesh.assign(freq_pos, freq_pos + n_freq);
    Geo& g = f->g;
    g.N = n_freq;
    g.Ns = lat->Ns;
    g.nc = lat->nc;
    g.npair = n_freq * (n_freq + 1) / 2;
    g.nmax = 2 * n_freq + 8;
    g.nent = (long)g.npair * n_freq * g.nc * g.Ns;
    g.nsp = (g.Ns + 3) & ~3;
    g.nentp = (long)g.npair * n_freq * g.nc * g.nsp;
    {
        const unsigned long long d = (unsigned long long)(g.nsp / 4);
        g.div4 = d > 1 ? (unsigned)((0x100000000ULL + d - 1) / d) : 0u;
    }
    if ((long)g.npair * n_freq * g.nc * g.Ns >= (1L << 31)) return fail(SR_EINVAL, "vertex too large for 32-bit offsets");

    // lattice tables
    std::vector<int> sp(lat->Ns), op(lat->Ns);
    for (int r = 0; r < lat->Ns; ++r) { sp[r] = pack_perm(lat->swap_perm[r]); op[r] = pack_perm(lat->onsite_perm[r]); }
    // lattice sum: distinct products (row index A, row index B) over all table entries and
    // components, and for every output (site, component) the list of its products
    std::vector<int2> prods;
    std::vector<int> goff(lat->Ns * lat->nc + 1, 0), gidx;
    if (lat->nc != 16) {
        std::map<std::pair<int, int>, int> pid;
        for (int r = 0; r < lat->Ns; ++r)
            for (int c = 0; c < lat->nc; ++c) {
                goff[r * lat->nc + c] = (int)gidx.size();
                for (int e = lat->rpa_off[r]; e < lat->rpa_off[r + 1]; ++e) {
                    const sr::RpaEntry& en = lat->rpa[e];
                    int ia = en.rA * lat->nc + en.pA[c], ib = en.rB * lat->nc + en.pB[c];
                    auto key = std::make_pair(ia, ib);
                    auto it = pid.find(key);
                    int u;
                    if (it == pid.end()) { u = (int)prods.size(); pid[key] = u; prods.push_back(make_int2(ia, ib)); }
                    else u = it->second;
                    gidx.push_back(u);
                }
            }
        goff[lat->Ns * lat->nc] = (int)gidx.size();
    }
    f->nprod = (int)prods.size();
    f->h_prod = prods;
    f->h_goff = goff;
    f->h_gidx = gidx;
    // padded-layout products, site-exchange map, dense (SU2) gather indices
    if (lat->nc != 16) {
        const int nsp = g.nsp;
        std::vector<int2> pp(prods.size());
        for (size_t k = 0; k < prods.size(); ++k) {
            const int ra = prods[k].x / lat->nc, ca = prods[k].x % lat->nc;
            const int rb = prods[k].y / lat->nc, cb = prods[k].y % lat->nc;
            pp[k] = make_int2(ca * nsp + ra, cb * nsp + rb);
        }
        CK(f->prodp.upload(pp.data(), pp.size(), f->stream));
        f->has_swap = false;
        for (int r = 0; r < lat->Ns; ++r) {
            if (lat->swap_r[r] != r) f->has_swap = true;
            for (int c = 0; c < lat->nc; ++c) if (lat->swap_perm[r][c] != c) f->has_swap = true;
        }
        f->dense = lat->nc == 2;
        std::vector<int> dg(gidx.size());
        for (size_t k = 0; k < gidx.size(); ++k) {
            const int ra = prods[gidx[k]].x / lat->nc, ca = prods[gidx[k]].x % lat->nc;
            const int rb = prods[gidx[k]].y / lat->nc;
            dg[k] = ca * nsp * nsp + ra * nsp + rb;
        }
        CK(f->dgath_idx.upload(dg.data(), dg.size(), f->stream));
    }
    std::vector<double> ih(n_freq - 1);
    for (int i = 0; i + 1 < n_freq; ++i) ih[i] = 1.0 / (freq_pos[i + 1] - freq_pos[i]);
    cudaStream_t st = f->stream;
    CK(f->w.upload(freq_pos, n_freq, st));
    CK(f->invh.upload(ih.data(), ih.size(), st));
    {
        std::vector<float> wfl(n_freq), ihf(n_freq - 1);
        for (int i = 0; i < n_freq; ++i) wfl[i] = (float)freq_pos[i];
        for (int i = 0; i + 1 < n_freq; ++i) ihf[i] = 1.0f / (wfl[i + 1] - wfl[i]);
        CK(f->wf.upload(wfl.data(), wfl.size(), st));
        CK(f->invhf.upload(ihf.data(), ihf.size(), st));
        g.log2w0 = (float)std::log2(freq_pos[0]);
        g.inv_dlog2 = (float)((n_freq - 1) / std::log2(freq_pos[n_freq - 1] / freq_pos[0]));
    }
    CK(f->swap_r.upload(lat->swap_r.data(), lat->Ns, st));
    CK(f->swap_perm.upload(sp.data(), lat->Ns, st));
    CK(f->onsite_perm.upload(op.data(), lat->Ns, st));
    CK(f->mult.upload(lat->mult.data(), lat->Ns, st));
    CK(f->prod.upload(prods.data(), prods.size(), st));
    CK(f->gath_off.upload(goff.data(), goff.size(), st));
    CK(f->gath_idx.upload(gidx.data(), gidx.size(), st));
    CK(f->init.upload(init_host.data(), init_host.size(), st));
    {
        std::vector<int2> cm(lat->chi_map.size());
        for (size_t i = 0; i < cm.size(); ++i) cm[i] = make_int2(lat->chi_map[i].r, pack_perm(lat->chi_map[i].perm));
        CK(f->chi_map.upload(cm.data(), cm.size(), st));
        CK(f->chi_onsite.upload(lat->chi_onsite.data(), lat->chi_onsite.size(), st));
        CK(f->chi_dr.upload(lat->chi_dr.data(), lat->chi_dr.size(), st));
        CK(f->chi.alloc(lat->chi_map.size() * g.nc * ts));
    }
    if (lat->nc == 16) {
        // TRI core: component maps and the lattice-sum table: per entry (rA, mA, rB, mB) of an
        // output site, the row indices and signs of A^{mu l} = (ref, j) and B^{l nu} = (j, i2);
        // work items split every site's entries into chunks, at most one item per thread of a
        // CTA when the table allows (items of a site are summed in a fixed order at the end)
        const int Ns = lat->Ns;
        std::vector<int> sm((size_t)Ns * 16), om((size_t)Ns * 16);
        for (int r = 0; r < Ns; ++r)
            for (int c = 0; c < 16; ++c) { sm[c * Ns + r] = lat->swap_map16[r][c]; om[r * 16 + c] = lat->onsite_map16[r][c]; }
        if (Ns * 16 > 0x7fff) return fail(SR_EUNSUPPORTED, "TRI lattice-sum table: too many irreducible sites (%d)", Ns);
        const long P = (long)lat->rpa16.size();
        std::vector<uint4> rec((size_t)P * 4);
        for (long e = 0; e < P; ++e) {
            const sr::RpaEntry16& en = lat->rpa16[e];
            unsigned code[32];
            for (int k = 0; k < 16; ++k) {
                code[k] = (unsigned)tri_slot(en.rA, en.mA[k] & 15);
                code[16 + k] = (unsigned)tri_slot(en.rB, en.mB[k] & 15);
            }
            // signs of signed permutations factorise: sign A^{mu l} = alpha(mu) beta(l),
            // sign B^{l nu} = gamma(l) delta(nu) (with beta(0) = gamma(0) = 1)
            auto sgn = [](int m) { return (m & 16) ? -1 : 1; };
            int alpha[4], beta[4], gamma_[4], delta[4];
            for (int l = 0; l < 4; ++l) { beta[l] = sgn(en.mA[0 * 4 + l]) * sgn(en.mA[0]); gamma_[l] = sgn(en.mB[l * 4 + 0]) * sgn(en.mB[0]); }
            for (int m = 0; m < 4; ++m) { alpha[m] = sgn(en.mA[m * 4 + 0]); delta[m] = sgn(en.mB[0 * 4 + m]); }
            for (int m = 0; m < 4; ++m)
                for (int l = 0; l < 4; ++l)
                    if (sgn(en.mA[m * 4 + l]) != alpha[m] * beta[l] || sgn(en.mB[l * 4 + m]) != gamma_[l] * delta[m])
                        return fail(SR_ESYMMETRY, "lattice-sum component map is not a signed permutation");
            for (int m = 0; m < 4; ++m) {
                if (alpha[m] < 0) code[m] |= 0x8000u;
                if (delta[m] < 0) code[4 + m] |= 0x8000u;
                if (beta[m] * gamma_[m] < 0) code[8 + m] |= 0x8000u;
            }
            unsigned wd[16];
            for (int k = 0; k < 16; ++k) wd[k] = code[2 * k] | (code[2 * k + 1] << 16);
            for (int v = 0; v < 4; ++v) rec[(size_t)e * 4 + v] = make_uint4(wd[4 * v], wd[4 * v + 1], wd[4 * v + 2], wd[4 * v + 3]);
        }
        const long per = std::max<long>(1, (P + (kThreads - Ns) - 1) / std::max(1, kThreads - Ns));
        std::vector<int4> items;
        std::vector<int> ioff((size_t)Ns + 1, 0);
        for (int r = 0; r < Ns; ++r) {
            ioff[r] = (int)items.size();
            for (int e = lat->rpa_off[r]; e < lat->rpa_off[r + 1]; e += (int)per)
                items.push_back(make_int4(r, e, (int)std::min<long>(e + per, lat->rpa_off[r + 1]), 0));
        }
        ioff[Ns] = (int)items.size();
        f->tlat_n_items = (int)items.size();
        if (precision == SR_FP64) {
            // FP64 kernel: per output (site, mu nu), every signed product of its entries
            std::vector<int> loff((size_t)Ns * 16 + 1, 0);
            std::vector<int2> lent;
            for (int r = 0; r < Ns; ++r)
                for (int c = 0; c < 16; ++c) {
                    loff[r * 16 + c] = (int)lent.size();
                    const int mu = c / 4, nu = c % 4;
                    for (int e = lat->rpa_off[r]; e < lat->rpa_off[r + 1]; ++e) {
                        const sr::RpaEntry16& en = lat->rpa16[e];
                        for (int l = 0; l < 4; ++l) {
                            const int ma = en.mA[mu * 4 + l], mb = en.mB[l * 4 + nu];
                            int sg = sr::tri::coef_t(mu, nu, l);
                            if (ma & 16) sg = -sg;
                            if (mb & 16) sg = -sg;
                            const int ia = tri_slot(en.rA, ma & 15), ib = tri_slot(en.rB, mb & 15);
                            lent.push_back(make_int2(ia, sg > 0 ? ib : ~ib));
                        }
                    }
                }
            loff[(size_t)Ns * 16] = (int)lent.size();
            CK(f->tlat_off.upload(loff.data(), loff.size(), st));
            CK(f->tlat_ent.upload(lent.data(), lent.size(), st));
        }
        CK(f->swap_map16.upload(sm.data(), sm.size(), st));
        CK(f->onsite_map16.upload(om.data(), om.size(), st));
        CK(f->tlat_rec.upload(rec.data(), rec.size(), st));
        CK(f->tlat_items.upload(items.data(), items.size(), st));
        CK(f->tlat_item_off.upload(ioff.data(), ioff.size(), st));
        std::vector<int> cr(lat->chi_map16.size()), cm(lat->chi_map16.size() * 16);
        for (size_t i = 0; i < cr.size(); ++i) {
            cr[i] = lat->chi_map16[i].r;
            for (int c = 0; c < 16; ++c) cm[i * 16 + c] = lat->chi_map16[i].m[c];
        }
        CK(f->chi_r16.upload(cr.data(), cr.size(), st));
        CK(f->chi_m16.upload(cm.data(), cm.size(), st));
        f->nprod = (int)(64 * P);   // products of the lattice sum per node (reported)
    }
    // state
    CK(f->gam.alloc((size_t)g.N * ts));
    CK(f->G.alloc((size_t)g.nent * ts));
    CK(f->dgam.alloc((size_t)g.N * ts));
    CK(f->dG.alloc((size_t)g.nent * ts));
    if (precision == SR_FP32_MIXED) CK(f->Gf.alloc(g.nc == 16 ? (size_t)g.nent : (size_t)g.nentp * (f->has_swap ? 2 : 1)));
    CK(f->nx.alloc((size_t)3 * g.N * g.nmax));
    CK(f->nW.alloc((size_t)3 * g.N * g.nmax * ts));
    CK(f->nWf.alloc((size_t)3 * g.N * g.nmax));
    CK(f->nxf.alloc((size_t)3 * g.N * g.nmax));
    CK(f->ncount.alloc((size_t)3 * g.N));
    CK(f->flag.alloc(1));
    CK(f->errbits.alloc(2));
    CK(cudaMemsetAsync(f->gam.p, 0, sizeof(double) * g.N * ts, st));
    if (f->ntan)
        k_fill_init<DualT><<<(unsigned)((g.nent + 255) / 256), 256, 0, st>>>(g, reinterpret_cast<const DualT*>(f->init.p),
                                                                            reinterpret_cast<DualT*>(f->G.p));
    else
        k_fill_init<double><<<(unsigned)((g.nent + 255) / 256), 256, 0, st>>>(g, f->init.p, f->G.p);
    CK(cudaGetLastError());
    if (sr_status s2 = refresh_shadow(f.get(), f->G.p, f->Gf.p)) return s2;
    const bool tc_ok = precision == SR_FP32_MIXED && tc_supported(g.nc, g.nsp, f->dense);
    f->smem_rhs = g.nc == 16 ? tri_smem_bytes(g.Ns, tri_groups(g.Ns, kThreads), f->tlat_n_items,
                                              precision == SR_FP64 ? (f->ntan ? sizeof(DualT) : sizeof(double)) : sizeof(float))
                  : precision == SR_FP32_MIXED ? f32_smem_bytes(g.Ns, g.nsp, g.nc, f->nprod, f->dense)
                                               : rhs_smem_bytes(g, f->nprod, f->ntan ? sizeof(DualT) : sizeof(double));
    if (tc_ok) f->smem_tc = f32_smem_bytes(g.Ns, g.nsp, g.nc, f->nprod, f->dense, true);
    f->use_tc = false;   // off by default: slower than the CUDA-core contraction on the square
                         // J1-J2 and pyrochlore workloads (operand staging outweighs the contraction)
    CK(f->tcfail.alloc(1));
    CK(cudaMemsetAsync(f->tcfail.p, 0, sizeof(int), st));
    if (f->smem_rhs > 227 * 1024) return fail(SR_EUNSUPPORTED, "lattice too large for one CTA's shared memory (%zu bytes)", f->smem_rhs);
    if (g.nc == 16) {
        if (f->ntan) CK(ensure_smem((const void*)k_gamma_rhs_tri<DualT>, f->smem_rhs));
        else if (precision == SR_FP64) CK(ensure_smem((const void*)k_gamma_rhs_tri<double>, f->smem_rhs));
        else CK(ensure_smem((const void*)k_gamma_rhs_tri<float>, f->smem_rhs));
    } else if (f->ntan) {
        CK(ensure_smem((const void*)k_gamma_rhs<DualT, 2>, f->smem_rhs));
        CK(ensure_smem((const void*)k_gamma_rhs<DualT, 4>, f->smem_rhs));
    } else if (precision == SR_FP64) {
        CK(ensure_smem((const void*)k_gamma_rhs<double, 2>, f->smem_rhs));
        CK(ensure_smem((const void*)k_gamma_rhs<double, 4>, f->smem_rhs));
    } else {
        CK(ensure_smem((const void*)k_gamma_rhs_f32<2, true>, f->smem_rhs));
        if (g.nc == 2 && f->dense && g.nsp / 2 <= su2f::kThreadsS) {
            // FP32-mixed SU2 kernel: the largest node block (64, 32, 16) whose shared memory
            // leaves room for the resident CTAs its registers allow, else the smallest that fits
            const int nth = su2f::threads_for(g.nsp);
            const int ctas = (su2f::cache_for(g.nsp) ? su2f::kMinCtasCached : su2f::kMinCtas) * su2f::kThreadsS / nth;
            for (int qb : {64, 32, 16}) {
                const size_t b = su2f::layout(g.N, g.Ns, g.nsp, qb, nth).total;
                if (b <= 227 * 1024 / ctas || (qb == 16 && b <= 227 * 1024)) { f->su2f_qb = qb; f->smem_su2f = b; break; }
            }
            if (f->su2f_qb > 0)
                CK(ensure_smem(su2f::cache_for(g.nsp) ? (const void*)k_gamma_rhs_su2f<true> : (const void*)k_gamma_rhs_su2f<false>,
                               f->smem_su2f));
        }
        CK(ensure_smem((const void*)k_gamma_rhs_f32<2, false>, f->smem_rhs));
        CK(ensure_smem((const void*)k_gamma_rhs_f32<4, false>, f->smem_rhs));
        if (tc_ok) {
            // persistent grid: resident CTAs per SM limited by the kernel's resources and by
            // the SM's 512 TMEM columns
            CK(ensure_smem((const void*)k_gamma_rhs_f32_tc, f->smem_tc));
            int occ = 0, dev = 0, nsm = 0, regs_sm = 0, smem_sm = 0, resv = 0;
            cudaFuncAttributes fa;
            CK(cudaFuncGetAttributes(&fa, k_gamma_rhs_f32_tc));
            CK(cudaGetDevice(&dev));
            CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            CK(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
            CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
            CK(cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev));
            const int regs = (fa.numRegs + 7) & ~7;
            occ = std::min(regs_sm / (regs * kThreads), (int)(smem_sm / (f->smem_tc + fa.sharedSizeBytes + resv)));
            occ = std::min(occ, 512 / tc_shape(g.nsp).ncols);
            f->tc_occ_api = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&f->tc_occ_api, k_gamma_rhs_f32_tc, kThreads, f->smem_tc));
            if (occ < 1) return fail(SR_EUNSUPPORTED, "tensor-core kernel cannot be resident (%zu bytes)", f->smem_tc);
            f->tc_grid = nsm * occ;
        }
    }
    CK(cudaStreamSynchronize(st));
    *out = f.release();
    return SR_OK;
}

extern "C" sr_status sr_flow_init(const sr_lattice* lat, int n_freq, const double* freq_pos, double lambda_init,
                                  sr_precision precision, void* cuda_stream, sr_flow** out) {
    return flow_create(lat, n_freq, freq_pos, lambda_init, precision, cuda_stream, 0, nullptr, out);
}

extern "C" sr_status sr_flow_init_tangent(const sr_lattice* lat, int n_freq, const double* freq_pos, double lambda_init,
                                          int n_par, const double* dM, void* cuda_stream, sr_flow** out) {
    if (n_par < 1 || n_par > kTan || !dM) return fail(SR_EINVAL, "n_par must be in [1, %d] with derivative couplings given", kTan);
    return flow_create(lat, n_freq, freq_pos, lambda_init, SR_FP64, cuda_stream, n_par, dM, out);
}

extern "C" sr_status sr_flow_set_tensor_cores(sr_flow* f, int on) {
    if (!f) return fail(SR_EINVAL, "null flow");
    if (on && !(f->prec == SR_FP32_MIXED && tc_supported(f->g.nc, f->g.nsp, f->dense)))
        return fail(SR_EUNSUPPORTED, "tensor-core lattice sum needs an FP32-mixed SU2 flow with at most 64 padded sites");
    f->use_tc = on != 0;
    return SR_OK;
}

extern "C" sr_status sr_flow_tensor_cores(const sr_flow* f, int* on) {
    if (!f || !on) return fail(SR_EINVAL, "null argument");
    *on = f->use_tc ? 1 : 0;
    return SR_OK;
}

extern "C" sr_status sr_flow_tangents(const sr_flow* f, int* n_tangent) {
    if (!f || !n_tangent) return fail(SR_EINVAL, "null argument");
    *n_tangent = f->ntan;
    return SR_OK;
}

extern "C" sr_status sr_flow_sizes(const sr_flow* f, long* n_gamma, int* n_freq, int* n_comp) {
    if (!f) return fail(SR_EINVAL, "null flow");
    if (n_gamma) *n_gamma = f->g.nent;
    if (n_freq) *n_freq = f->g.N;
    if (n_comp) *n_comp = f->g.nc;
    return SR_OK;
}

extern "C" sr_status sr_flow_rhs(sr_flow* f, double lambda, double* d_dsigma, double* d_dgamma) {
    if (!f) return fail(SR_EINVAL, "null flow");
    if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(SR_EINVAL, "lambda must be positive");
    if (sr_status s = run_rhs(f, lambda, f->gam.p, f->G.p, f->Gf.p, f->dgam.p, f->dG.p)) return s;
    if (d_dsigma) CK(cudaMemcpyAsync(d_dsigma, f->dgam.p, sizeof(double) * f->g.N * f->ts, cudaMemcpyDeviceToDevice, f->stream));
    if (d_dgamma) CK(cudaMemcpyAsync(d_dgamma, f->dG.p, sizeof(double) * f->g.nent * f->ts, cudaMemcpyDeviceToDevice, f->stream));
    return SR_OK;
}

static sr_status check_flag(sr_flow* f, double lam) {
    int h = 0, t = 0;
    CK(cudaMemcpyAsync(&h, f->flag.p, sizeof(int), cudaMemcpyDeviceToHost, f->stream));
    CK(cudaMemcpyAsync(&t, f->tcfail.p, sizeof(int), cudaMemcpyDeviceToHost, f->stream));
    CK(cudaStreamSynchronize(f->stream));
    if (t) return fail(SR_ETIMEOUT, "tensor-core MMA completion wait gave up (Lambda = %.17g)", lam);
    if (h) return fail(SR_ENONFINITE, "non-finite value in the flow at Lambda = %.17g", lam);
    return SR_OK;
}

static sr_status euler_step(sr_flow* f, double lam_next) {
    const Geo& g = f->g;
    const double dl = f->lambda - lam_next;
    if (sr_status s = run_rhs(f, f->lambda, f->gam.p, f->G.p, f->Gf.p, f->dgam.p, f->dG.p)) return s;
    CK(cudaMemsetAsync(f->flag.p, 0, sizeof(int), f->stream));
    const long nG = g.nent * f->ts;
    k_axpy<<<1, 256, 0, f->stream>>>((long)g.N * f->ts, f->gam.p, f->dgam.p, -dl, f->flag.p);
    k_axpy<<<(unsigned)((nG + 255) / 256), 256, 0, f->stream>>>(nG, f->G.p, f->dG.p, -dl, f->flag.p);
    CK(cudaGetLastError());
    if (sr_status s = refresh_shadow(f, f->G.p, f->Gf.p)) return s;
    if (sr_status s = check_flag(f, lam_next)) return s;
    f->lambda = lam_next;
    return SR_OK;
}

// ----------------------------------------------------------------------------- sharded right-hand side

extern "C" sr_status sr_flow_rhs_pairs(sr_flow* f, double lambda, int pair_begin, int pair_end, double* d_dsigma,
                                       double* d_dgamma) {
    if (!f) return fail(SR_EINVAL, "null flow");
    if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(SR_EINVAL, "lambda must be positive");
    if (pair_begin < 0 || pair_end < pair_begin || pair_end > f->g.npair)
        return fail(SR_EINVAL, "pair range [%d, %d) outside [0, %d]", pair_begin, pair_end, f->g.npair);
    if (!d_dsigma || !d_dgamma) return fail(SR_EINVAL, "null output");
    // the vertex kernels write only the range's slice of the state layout, straight into d_dgamma
    if (sr_status s = run_rhs(f, lambda, f->gam.p, f->G.p, f->Gf.p, d_dsigma, d_dgamma, pair_begin, pair_end)) return s;
    return SR_OK;
}

extern "C" sr_status sr_flow_advance(sr_flow* f, double lambda_next, const double* d_dsigma, const double* d_dgamma) {
    if (!f) return fail(SR_EINVAL, "null flow");
    if (!d_dsigma || !d_dgamma) return fail(SR_EINVAL, "null right-hand side");
    if (!(lambda_next > 0.0) || !(lambda_next < f->lambda)) return fail(SR_EINVAL, "lambda_next must lie in (0, lambda)");
    const Geo& g = f->g;
    const double dl = f->lambda - lambda_next;
    CK(cudaMemsetAsync(f->flag.p, 0, sizeof(int), f->stream));
    const long nG = g.nent * f->ts;
    k_axpy<<<1, 256, 0, f->stream>>>((long)g.N * f->ts, f->gam.p, d_dsigma, -dl, f->flag.p);
    k_axpy<<<(unsigned)((nG + 255) / 256), 256, 0, f->stream>>>(nG, f->G.p, d_dgamma, -dl, f->flag.p);
    CK(cudaGetLastError());
    if (sr_status s = refresh_shadow(f, f->G.p, f->Gf.p)) return s;
    if (sr_status s = check_flag(f, lambda_next)) return s;
    f->lambda = lambda_next;
    f->fsal = false;
    return SR_OK;
}

static sr_status ensure_rk(sr_flow* f) {
    if (f->y0G.p) return SR_OK;
    const Geo& g = f->g;
    CK(f->y0g.alloc(g.N));
    CK(f->y0G.alloc(g.nent));
    CK(f->stg.alloc(g.N));
    CK(f->stG.alloc(g.nent));
    for (int i = 0; i < 7; ++i) { CK(f->kg[i].alloc(g.N)); CK(f->kG[i].alloc(g.nent)); }
    return SR_OK;
}

// One Dormand-Prince 5(4) step of size h from the current state; writes the fifth-order
// solution into the state and the error norm into f->last_err (synchronises).
static sr_status dp54_step(sr_flow* f, double h, double rtol, double atol) {
    static const double C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
    static const double A[7][6] = {{0},
                                   {1.0 / 5},
                                   {3.0 / 40, 9.0 / 40},
                                   {44.0 / 45, -56.0 / 15, 32.0 / 9},
                                   {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729},
                                   {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656},
                                   {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
    if (sr_status s = ensure_rk(f)) return s;
    const Geo& g = f->g;
    cudaStream_t st = f->stream;
    CK(cudaMemcpyAsync(f->y0g.p, f->gam.p, sizeof(double) * g.N, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(f->y0G.p, f->G.p, sizeof(double) * g.nent, cudaMemcpyDeviceToDevice, st));
    KPtrs pg, pG;
    for (int i = 0; i < 7; ++i) { pg.k[i] = f->kg[i].p; pG.k[i] = f->kG[i].p; }
    const unsigned bG = (unsigned)((g.nent + 255) / 256);
    for (int s = 0; s < 7; ++s) {
        const double* sg = f->y0g.p;
        const double* sG = f->y0G.p;
        if (s == 0 && f->fsal) {
            // first-same-as-last: the last stage of the previous accepted step is this step's first
            std::swap(f->kg[0].p, f->kg[6].p);
            std::swap(f->kG[0].p, f->kG[6].p);
            pg.k[0] = f->kg[0].p; pg.k[6] = f->kg[6].p;
            pG.k[0] = f->kG[0].p; pG.k[6] = f->kG[6].p;
            continue;
        }
        if (s > 0) {
            k_rk_stage<<<1, 256, 0, st>>>(g.N, f->y0g.p, pg, s, A[s][0], A[s][1], A[s][2], A[s][3], A[s][4], A[s][5], h, f->stg.p);
            k_rk_stage<<<bG, 256, 0, st>>>(g.nent, f->y0G.p, pG, s, A[s][0], A[s][1], A[s][2], A[s][3], A[s][4], A[s][5], h, f->stG.p);
            CK(cudaGetLastError());
            sg = f->stg.p;
            sG = f->stG.p;
        }
        if (sr_status e = refresh_shadow(f, sG, f->Gf.p)) return e;
        if (sr_status e = run_rhs(f, f->lambda + C[s] * h, sg, sG, f->Gf.p, f->kg[s].p, f->kG[s].p)) return e;
    }
    CK(cudaMemsetAsync(f->errbits.p, 0, 2 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(f->flag.p, 0, sizeof(int), st));
    k_rk_final<<<1, 256, 0, st>>>(g.N, f->y0g.p, pg, h, f->gam.p, f->errbits.p, f->flag.p);
    k_rk_final<<<bG, 256, 0, st>>>(g.nent, f->y0G.p, pG, h, f->G.p, f->errbits.p, f->flag.p);
    CK(cudaGetLastError());
    unsigned long long eb[2] = {0, 0};
    int fl = 0;
    CK(cudaMemcpyAsync(eb, f->errbits.p, sizeof(eb), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&fl, f->flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double emax, ymax;
    std::memcpy(&emax, &eb[0], sizeof(double));
    std::memcpy(&ymax, &eb[1], sizeof(double));
    // normwise scaled error: max_i |e_i| / (atol + rtol max_i max(|y0_i|, |y_new_i|))
    f->last_err = emax / (atol + rtol * ymax);
    if (fl) return fail(SR_ENONFINITE, "non-finite value in a Dormand-Prince step at Lambda = %.17g", f->lambda);
    return SR_OK;
}

static sr_status restore_y0(sr_flow* f) {
    const Geo& g = f->g;
    CK(cudaMemcpyAsync(f->gam.p, f->y0g.p, sizeof(double) * g.N, cudaMemcpyDeviceToDevice, f->stream));
    CK(cudaMemcpyAsync(f->G.p, f->y0G.p, sizeof(double) * g.nent, cudaMemcpyDeviceToDevice, f->stream));
    return refresh_shadow(f, f->G.p, f->Gf.p);
}

extern "C" sr_status sr_flow_step(sr_flow* f, double lambda_next, int method, double rtol, double atol, double* reached) {
    if (!f) return fail(SR_EINVAL, "null flow");
    if (!(lambda_next > 0.0) || !(lambda_next < f->lambda)) return fail(SR_EINVAL, "lambda_next must lie in (0, lambda)");
    if (method == SR_EULER) {
        f->fsal = false;
        if (sr_status s = euler_step(f, lambda_next)) return s;
    } else if (f->ntan) {
        return fail(SR_EUNSUPPORTED, "tangent flows step with SR_EULER only");
    } else if (method == SR_RK_FIXED) {
        if (sr_status s = dp54_step(f, lambda_next - f->lambda, rtol, atol)) { f->fsal = false; return s; }
        if (sr_status s = refresh_shadow(f, f->G.p, f->Gf.p)) return s;
        f->lambda = lambda_next;
        f->fsal = true;
        f->n_accept++;
    } else if (method == SR_RK_ADAPTIVE) {
        if (!(rtol > 0.0) || !(atol >= 0.0)) return fail(SR_EINVAL, "rtol must be positive and atol non-negative");
        // step-size control (Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4, with the
        // stabilised PI variant for DOPRI5): accepted steps scale h by
        // 0.9 err^-0.17 err_prev^0.04 within [0.2, 5], never growing right after a rejection;
        // rejected steps by max(0.2, 0.9 err^-0.2).  A step cut short to land on lambda_next
        // does not shrink the proposal for the next call.
        double h = f->h_next < 0.0 ? f->h_next : (lambda_next - f->lambda);
        long guard = 0;
        bool rejected = false;
        while (f->lambda > lambda_next) {
            if (++guard > f->step_limit) {
                if (reached) *reached = f->lambda;
                return fail(SR_ETIMEOUT, "adaptive stepping stopped at Lambda = %.17g after %ld attempted steps",
                            f->lambda, f->step_limit);
            }
            const double h_prop = h;
            const bool cut = f->lambda + h < lambda_next;
            if (cut) h = lambda_next - f->lambda;
            sr_status s = dp54_step(f, h, rtol, atol);
            if (s != SR_OK && s != SR_ENONFINITE) return s;
            double err = s == SR_ENONFINITE ? INFINITY : f->last_err;
            if (err <= 1.0) {
                f->fsal = true;
                f->lambda += h;
                if (std::fabs(f->lambda - lambda_next) <= 1e-14 * std::fabs(lambda_next)) f->lambda = lambda_next;
                if (sr_status e = refresh_shadow(f, f->G.p, f->Gf.p)) return e;
                f->n_accept++;
                double fac = err == 0.0 ? 5.0 : 0.9 * std::pow(err, -0.17) * std::pow(f->err_prev, 0.04);
                fac = std::min(rejected ? 1.0 : 5.0, std::max(0.2, fac));
                f->err_prev = std::max(err, 1e-4);
                h = cut ? h_prop : h * fac;
                f->h_next = h;
                rejected = false;
            } else {
                const double fac = 0.9 * std::pow(err, -0.2);
                if (sr_status e = restore_y0(f)) return e;
                // the first stage (the right-hand side at the step's start) stays valid: park it
                // where the next attempt's first-same-as-last exchange picks it up
                std::swap(f->kg[0].p, f->kg[6].p);
                std::swap(f->kG[0].p, f->kG[6].p);
                f->fsal = true;
                f->n_reject++;
                rejected = true;
                h *= std::max(0.2, std::min(1.0, fac));
                if (std::fabs(h) < 1e-14 * f->lambda) return fail(SR_ENONFINITE, "step size underflow at Lambda = %.17g", f->lambda);
            }
        }
    } else {
        return fail(SR_EINVAL, "unknown method");
    }
    if (reached) *reached = f->lambda;
    return SR_OK;
}

extern "C" sr_status sr_flow_set_step_limit(sr_flow* f, long max_steps) {
    if (!f || max_steps <= 0) return fail(SR_EINVAL, "step limit must be positive");
    f->step_limit = max_steps;
    return SR_OK;
}

extern "C" sr_status sr_flow_stats(const sr_flow* f, double* last_err, long* n_rhs, long* n_accept, long* n_reject) {
    if (!f) return fail(SR_EINVAL, "null flow");
    if (last_err) *last_err = f->last_err;
    if (n_rhs) *n_rhs = f->n_rhs;
    if (n_accept) *n_accept = f->n_accept;
    if (n_reject) *n_reject = f->n_reject;
    return SR_OK;
}

extern "C" sr_status sr_measure_susceptibility_tangent(sr_flow* f, int n_k, const double* k_xyz, double* chi_k,
                                                      double* dchi_k) {
    if (!f || n_k <= 0 || !k_xyz || !chi_k || !dchi_k) return fail(SR_EINVAL, "bad arguments");
    if (!f->ntan) return fail(SR_EINVAL, "not a tangent flow (sr_flow_init_tangent)");
    const sr_lattice* lat = f->lat;
    const Geo& g = f->g;
    const int npairs = (int)lat->chi_map.size();
    Tabs tb = f->tabs();
    DualT* chi = reinterpret_cast<DualT*>(f->chi.p);
    if (g.nc == 16)
        k_chi_tri<DualT><<<npairs, 128, 0, f->stream>>>(g, tb, f->tabs_tri(), f->w.p, reinterpret_cast<const DualT*>(f->gam.p),
                                                        reinterpret_cast<const DualT*>(f->G.p), f->lambda, f->chi_r16.p,
                                                        f->chi_m16.p, f->chi_onsite.p, lat->Ntot, chi);
    else if (g.nc == 2)
        k_chi<DualT, 2><<<npairs, 128, 0, f->stream>>>(g, tb, f->w.p, reinterpret_cast<const DualT*>(f->gam.p),
                                                        reinterpret_cast<const DualT*>(f->G.p), f->lambda, f->chi_map.p,
                                                        f->chi_onsite.p, lat->Ntot, chi);
    else
        k_chi<DualT, 4><<<npairs, 128, 0, f->stream>>>(g, tb, f->w.p, reinterpret_cast<const DualT*>(f->gam.p),
                                                        reinterpret_cast<const DualT*>(f->G.p), f->lambda, f->chi_map.p,
                                                        f->chi_onsite.p, lat->Ntot, chi);
    CK(cudaGetLastError());
    if (f->kbuf.n < (size_t)3 * n_k) CK(f->kbuf.alloc((size_t)3 * n_k));
    if (f->chik.n < (size_t)n_k * f->ts) CK(f->chik.alloc((size_t)n_k * f->ts));
    CK(cudaMemcpyAsync(f->kbuf.p, k_xyz, sizeof(double) * 3 * n_k, cudaMemcpyHostToDevice, f->stream));
    if (g.nc == 16)
        k_chi_k_tri<DualT><<<(n_k + 127) / 128, 128, 0, f->stream>>>(n_k, f->kbuf.p, chi, f->chi_dr.p, npairs, lat->nb,
                                                                     reinterpret_cast<DualT*>(f->chik.p));
    else
        k_chi_k<DualT><<<(n_k + 127) / 128, 128, 0, f->stream>>>(n_k, f->kbuf.p, chi, f->chi_dr.p, npairs, lat->nb, g.nc,
                                                                 reinterpret_cast<DualT*>(f->chik.p));
    CK(cudaGetLastError());
    std::vector<double> h((size_t)n_k * f->ts);
    CK(cudaMemcpyAsync(h.data(), f->chik.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, f->stream));
    CK(cudaStreamSynchronize(f->stream));
    for (int i = 0; i < n_k; ++i) {
        chi_k[i] = h[(size_t)i * f->ts];
        for (int p = 0; p < f->ntan; ++p) dchi_k[(size_t)i * f->ntan + p] = h[(size_t)i * f->ts + 1 + p];
    }
    return SR_OK;
}

extern "C" sr_status sr_measure_susceptibility(sr_flow* f, int n_k, const double* k_xyz, double* chi_k, double* chi_ij) {
    if (!f) return fail(SR_EINVAL, "null flow");
    if (f->ntan) return fail(SR_EINVAL, "tangent flows measure with sr_measure_susceptibility_tangent");
    if (n_k < 0 || (n_k > 0 && chi_k && !k_xyz)) return fail(SR_EINVAL, "bad momenta");
    const sr_lattice* lat = f->lat;
    const Geo& g = f->g;
    const int npairs = (int)lat->chi_map.size();
    Tabs tb = f->tabs();
    if (g.nc == 16)
        k_chi_tri<<<npairs, 128, 0, f->stream>>>(g, tb, f->tabs_tri(), f->w.p, f->gam.p, f->G.p, f->lambda, f->chi_r16.p, f->chi_m16.p,
                                                 f->chi_onsite.p, lat->Ntot, f->chi.p);
    else if (g.nc == 2)
        k_chi<double, 2><<<npairs, 128, 0, f->stream>>>(g, tb, f->w.p, f->gam.p, f->G.p, f->lambda, f->chi_map.p, f->chi_onsite.p, lat->Ntot, f->chi.p);
    else
        k_chi<double, 4><<<npairs, 128, 0, f->stream>>>(g, tb, f->w.p, f->gam.p, f->G.p, f->lambda, f->chi_map.p, f->chi_onsite.p, lat->Ntot, f->chi.p);
    CK(cudaGetLastError());
    if (chi_ij) CK(cudaMemcpyAsync(chi_ij, f->chi.p, sizeof(double) * npairs * g.nc, cudaMemcpyDeviceToDevice, f->stream));
    if (chi_k && n_k > 0) {
        if (f->kbuf.n < (size_t)3 * n_k) CK(f->kbuf.alloc((size_t)3 * n_k));
        if (f->chik.n < (size_t)n_k) CK(f->chik.alloc(n_k));
        CK(cudaMemcpyAsync(f->kbuf.p, k_xyz, sizeof(double) * 3 * n_k, cudaMemcpyHostToDevice, f->stream));
        if (g.nc == 16)
            k_chi_k_tri<<<(n_k + 127) / 128, 128, 0, f->stream>>>(n_k, f->kbuf.p, f->chi.p, f->chi_dr.p, npairs, lat->nb, f->chik.p);
        else
            k_chi_k<double><<<(n_k + 127) / 128, 128, 0, f->stream>>>(n_k, f->kbuf.p, f->chi.p, f->chi_dr.p, npairs, lat->nb, g.nc, f->chik.p);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(chi_k, f->chik.p, sizeof(double) * n_k, cudaMemcpyDeviceToHost, f->stream));
        CK(cudaStreamSynchronize(f->stream));
    }
    return SR_OK;
}

// ----------------------------------------------------------------------------- adjoint
//
// Reverse-mode derivatives of the FP64 flow (plain, non-tangent flows): the transpose of the
// right-hand side's Jacobian at the current state, the transpose of one Euler step, and the
// gradient of a weighted sum of chi(k) with respect to the state.  The caller keeps (or
// recomputes from checkpoints) the forward states and sets each with sr_flow_set_state.

static sr_status adj_prepare(sr_flow* f) {
    if (f->adj_ready) return SR_OK;
    const Geo& g = f->g;
    if (g.nc == 16) {
        // TRI: the vertex adjoint walks the forward lattice-sum table itself
        CK(f->ntw.alloc((size_t)3 * g.N * g.nmax));
        CK(f->Wbar.alloc((size_t)3 * g.N * g.nmax));
        CK(f->dgbar.alloc((size_t)g.N));
        CK(f->tg.alloc((size_t)g.N));
        CK(f->tG.alloc((size_t)g.nent));
        f->smem_adj = tri_adj_smem_bytes(g.Ns);
        if (f->smem_adj > 227 * 1024) return fail(SR_EUNSUPPORTED, "lattice too large for the adjoint kernel (%zu bytes)", f->smem_adj);
        CK(ensure_smem((const void*)k_gamma_adj_tri, f->smem_adj));
        CK(cudaStreamSynchronize(f->stream));
        f->adj_ready = true;
        return SR_OK;
    }
    const int row = g.Ns * g.nc, np = f->nprod;
    std::vector<int> poff(np + 1, 0), pout(f->h_gidx.size());
    for (int o = 0; o < row; ++o)
        for (int k = f->h_goff[o]; k < f->h_goff[o + 1]; ++k) poff[f->h_gidx[k] + 1]++;
    for (int i = 0; i < np; ++i) poff[i + 1] += poff[i];
    {
        std::vector<int> fill(poff.begin(), poff.end() - 1);
        for (int o = 0; o < row; ++o)
            for (int k = f->h_goff[o]; k < f->h_goff[o + 1]; ++k) pout[fill[f->h_gidx[k]]++] = o;
    }
    std::vector<int> aoff(row + 1, 0), aidx(np), boff(row + 1, 0), bidx(np);
    for (int i = 0; i < np; ++i) { aoff[f->h_prod[i].x + 1]++; boff[f->h_prod[i].y + 1]++; }
    for (int e = 0; e < row; ++e) { aoff[e + 1] += aoff[e]; boff[e + 1] += boff[e]; }
    {
        std::vector<int> fa(aoff.begin(), aoff.end() - 1), fb(boff.begin(), boff.end() - 1);
        for (int i = 0; i < np; ++i) { aidx[fa[f->h_prod[i].x]++] = i; bidx[fb[f->h_prod[i].y]++] = i; }
    }
    cudaStream_t st = f->stream;
    auto up = [&](DevBuf<int>& b, const std::vector<int>& v) { return v.empty() ? b.alloc(1) : b.upload(v.data(), v.size(), st); };
    CK(up(f->pinv_off, poff));
    CK(up(f->pinv_out, pout));
    CK(up(f->ainv_off, aoff));
    CK(up(f->ainv_idx, aidx));
    CK(up(f->binv_off, boff));
    CK(up(f->binv_idx, bidx));
    CK(f->ntw.alloc((size_t)3 * g.N * g.nmax));
    CK(f->Wbar.alloc((size_t)3 * g.N * g.nmax));
    CK(f->dgbar.alloc((size_t)g.N));
    CK(f->tg.alloc((size_t)g.N));
    CK(f->tG.alloc((size_t)g.nent));
    f->smem_adj = adj_smem_bytes(g.Ns, g.nc, np);
    if (f->smem_adj > 227 * 1024) return fail(SR_EUNSUPPORTED, "lattice too large for the adjoint kernel (%zu bytes)", f->smem_adj);
    CK(ensure_smem(g.nc == 2 ? (const void*)k_gamma_adj<2> : (const void*)k_gamma_adj<4>, f->smem_adj));
    CK(cudaStreamSynchronize(st));
    f->adj_ready = true;
    return SR_OK;
}

static sr_status adj_check(const sr_flow* f) {
    if (!f) return fail(SR_EINVAL, "null flow");
    if (f->ntan) return fail(SR_EUNSUPPORTED, "the adjoint is defined for plain flows, not tangent flows");
    if (f->prec != SR_FP64) return fail(SR_EUNSUPPORTED, "the adjoint is defined for FP64 flows");
    return SR_OK;
}

// (gbar_o, Gbar_o) = J^T (fbar_g, fbar_G) at the current state and cutoff lam.
static sr_status rhs_adjoint(sr_flow* f, double lam, const double* fbar_g, const double* fbar_G, double* gbar_o,
                             double* Gbar_o) {
    if (sr_status s = adj_prepare(f)) return s;
    const Geo& g = f->g;
    Tabs tb = f->tabs();
    AdjTabs at{f->pinv_off.p, f->pinv_out.p, f->ainv_off.p, f->ainv_idx.p, f->binv_off.p, f->binv_idx.p};
    cudaStream_t st = f->stream;
    // forward quantities the derivatives need: dgamma, the node positions and weights
    if (g.nc == 16)
        k_sigma_rhs_tri<double><<<g.N, 64, 0, st>>>(g, tb, f->tabs_tri(), f->w.p, f->gam.p, f->G.p, lam, f->dgam.p);
    else
        k_sigma_rhs<double><<<g.N, 64, 0, st>>>(g, tb, f->w.p, f->gam.p, f->G.p, lam, f->dgam.p);
    k_channel_nodes<double><<<3 * g.N, 128, 0, st>>>(g, f->w.p, f->invh.p, f->gam.p, f->dgam.p, lam, f->nx.p, f->nW.p,
                                                     nullptr, f->ncount.p, nullptr, f->ntw.p);
    CK(cudaMemsetAsync(gbar_o, 0, sizeof(double) * g.N, st));
    CK(cudaMemsetAsync(Gbar_o, 0, sizeof(double) * g.nent, st));
    CK(cudaMemsetAsync(f->Wbar.p, 0, sizeof(double) * 3 * g.N * g.nmax, st));
    CK(cudaMemsetAsync(f->dgbar.p, 0, sizeof(double) * g.N, st));
    const int blocks = g.npair * g.N;
    if (g.nc == 16)
        k_gamma_adj_tri<<<blocks, kThreads, f->smem_adj, st>>>(g, tb, f->tabs_tri(), f->w.p, f->G.p, f->nx.p, f->nW.p,
                                                               f->ncount.p, fbar_G, Gbar_o, f->Wbar.p);
    else if (g.nc == 2)
        k_gamma_adj<2><<<blocks, kThreads, f->smem_adj, st>>>(g, tb, at, f->w.p, f->G.p, f->nx.p, f->nW.p, f->ncount.p,
                                                              fbar_G, Gbar_o, f->Wbar.p);
    else
        k_gamma_adj<4><<<blocks, kThreads, f->smem_adj, st>>>(g, tb, at, f->w.p, f->G.p, f->nx.p, f->nW.p, f->ncount.p,
                                                              fbar_G, Gbar_o, f->Wbar.p);
    k_nodes_adj<<<3 * g.N, 128, 0, st>>>(g, f->w.p, f->invh.p, f->gam.p, f->dgam.p, lam, f->nx.p, f->ntw.p, f->ncount.p,
                                         f->Wbar.p, gbar_o, f->dgbar.p);
    k_axmy<<<1, 256, 0, st>>>((long)g.N, f->dgbar.p, fbar_g, -1.0, f->dgbar.p);
    if (g.nc == 16)
        k_sigma_adj_tri<<<g.N, 64, 0, st>>>(g, tb, f->tabs_tri(), f->w.p, f->gam.p, f->G.p, lam, f->dgbar.p, gbar_o, Gbar_o);
    else
        k_sigma_adj<<<g.N, 64, 0, st>>>(g, tb, f->w.p, f->gam.p, f->G.p, lam, f->dgbar.p, gbar_o, Gbar_o);
    CK(cudaGetLastError());
    return SR_OK;
}

extern "C" sr_status sr_flow_rhs_adjoint(sr_flow* f, double lambda, const double* d_fbar_sigma, const double* d_fbar_gamma,
                                         double* d_bar_sigma, double* d_bar_gamma) {
    if (sr_status s = adj_check(f)) return s;
    if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(SR_EINVAL, "lambda must be positive");
    if (!d_fbar_sigma || !d_fbar_gamma || !d_bar_sigma || !d_bar_gamma) return fail(SR_EINVAL, "null buffer");
    return rhs_adjoint(f, lambda, d_fbar_sigma, d_fbar_gamma, d_bar_sigma, d_bar_gamma);
}

extern "C" sr_status sr_flow_step_adjoint(sr_flow* f, double lambda_from, double lambda_to, const double* d_bar_sigma_in,
                                          const double* d_bar_gamma_in, double* d_bar_sigma_out, double* d_bar_gamma_out) {
    if (sr_status s = adj_check(f)) return s;
    if (!d_bar_sigma_in || !d_bar_gamma_in || !d_bar_sigma_out || !d_bar_gamma_out) return fail(SR_EINVAL, "null buffer");
    if (!(lambda_from > 0.0) || !(lambda_to > 0.0) || !std::isfinite(lambda_from) || !std::isfinite(lambda_to))
        return fail(SR_EINVAL, "cutoffs must be positive");
    if (f->lambda != lambda_from)
        return fail(SR_EINVAL, "the flow's state is at Lambda = %.17g, not at lambda_from = %.17g", f->lambda, lambda_from);
    if (sr_status s = adj_prepare(f)) return s;
    const Geo& g = f->g;
    if (sr_status s = rhs_adjoint(f, lambda_from, d_bar_sigma_in, d_bar_gamma_in, f->tg.p, f->tG.p)) return s;
    const double dl = lambda_from - lambda_to;
    k_axmy<<<1, 256, 0, f->stream>>>((long)g.N, d_bar_sigma_in, f->tg.p, dl, d_bar_sigma_out);
    k_axmy<<<(unsigned)((g.nent + 255) / 256), 256, 0, f->stream>>>(g.nent, d_bar_gamma_in, f->tG.p, dl, d_bar_gamma_out);
    CK(cudaGetLastError());
    return SR_OK;
}

extern "C" sr_status sr_measure_susceptibility_adjoint(sr_flow* f, int n_k, const double* k_xyz, const double* chi_bar,
                                                       double* d_bar_sigma, double* d_bar_gamma) {
    if (sr_status s = adj_check(f)) return s;
    if (n_k <= 0 || !k_xyz || !chi_bar || !d_bar_sigma || !d_bar_gamma) return fail(SR_EINVAL, "bad arguments");
    const sr_lattice* lat = f->lat;
    const Geo& g = f->g;
    const int npairs = (int)lat->chi_map.size();
    cudaStream_t st = f->stream;
    if (f->kbar.n < (size_t)4 * n_k) CK(f->kbar.alloc((size_t)4 * n_k));
    if (f->chibar.n < (size_t)npairs * g.nc) CK(f->chibar.alloc((size_t)npairs * g.nc));
    CK(cudaMemcpyAsync(f->kbar.p, k_xyz, sizeof(double) * 3 * n_k, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(f->kbar.p + 3 * n_k, chi_bar, sizeof(double) * n_k, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(d_bar_sigma, 0, sizeof(double) * g.N, st));
    CK(cudaMemsetAsync(d_bar_gamma, 0, sizeof(double) * g.nent, st));
    Tabs tb = f->tabs();
    if (g.nc == 16) {
        k_chik_adj_tri<<<(npairs + 127) / 128, 128, 0, st>>>(n_k, f->kbar.p, f->kbar.p + 3 * n_k, f->chi_dr.p, npairs, lat->nb,
                                                             f->chibar.p);
        k_chi_adj_tri<<<npairs, 128, 0, st>>>(g, tb, f->tabs_tri(), f->w.p, f->gam.p, f->G.p, f->lambda, f->chi_r16.p,
                                              f->chi_m16.p, f->chi_onsite.p, lat->Ntot, f->chibar.p, d_bar_sigma, d_bar_gamma);
    } else {
        k_chik_adj<<<(npairs + 127) / 128, 128, 0, st>>>(n_k, f->kbar.p, f->kbar.p + 3 * n_k, f->chi_dr.p, npairs, lat->nb,
                                                         g.nc, f->chibar.p);
        if (g.nc == 2)
            k_chi_adj<2><<<npairs, 128, 0, st>>>(g, tb, f->w.p, f->gam.p, f->G.p, f->lambda, f->chi_map.p, f->chi_onsite.p,
                                                 lat->Ntot, f->chibar.p, d_bar_sigma, d_bar_gamma);
        else
            k_chi_adj<4><<<npairs, 128, 0, st>>>(g, tb, f->w.p, f->gam.p, f->G.p, f->lambda, f->chi_map.p, f->chi_onsite.p,
                                                 lat->Ntot, f->chibar.p, d_bar_sigma, d_bar_gamma);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return SR_OK;
}

// ----------------------------------------------------------------------------- coupling parameters

extern "C" sr_status sr_couplings_linear(int n_par, const double* theta, int n_couplings, const double* B, double* M) {
    if (n_par < 1 || n_couplings < 0 || !theta || (n_couplings > 0 && (!B || !M))) return fail(SR_EINVAL, "bad arguments");
    for (int c = 0; c < n_couplings; ++c)
        for (int e = 0; e < 9; ++e) {
            double acc = 0.0;
            for (int q = 0; q < n_par; ++q) acc += theta[q] * B[((size_t)q * n_couplings + c) * 9 + e];
            M[(size_t)c * 9 + e] = acc;
        }
    return SR_OK;
}

namespace {
// Column sums of the state-layout array a over all stored frequency triples: out[c * Ns + r] =
// sum over (pair, t) of a[((pair N + t) nc + c) Ns + r]; one block per (c, r), fixed reduction
// order.
__global__ void k_entry_column_sum(Geo g, const double* __restrict__ a, double* __restrict__ out) {
    __shared__ double red[32];
    const int cr = blockIdx.x, row = g.nc * g.Ns;
    const long ntrip = (long)g.npair * g.N;
    double acc[1] = {0.0};
    for (long i = threadIdx.x; i < ntrip; i += blockDim.x) acc[0] += a[i * row + cr];
    block_sum<double, 1>(acc, red);
    if (threadIdx.x == 0) out[(cr % g.Ns) * g.nc + cr / g.Ns] = acc[0];
}
}  // namespace

extern "C" sr_status sr_flow_initial_vertex_adjoint(sr_flow* f, int n_par, const double* dM, const double* d_bar_gamma,
                                                   double* grad) {
    if (!f || n_par < 1 || !dM || !d_bar_gamma || !grad) return fail(SR_EINVAL, "bad arguments");
    if (f->ntan) return fail(SR_EUNSUPPORTED, "plain flows only (not tangent flows)");
    const Geo& g = f->g;
    std::vector<double> dinit;
    std::string msg;
    if (sr_status s = sr::tangent_init(f->lat, n_par, dM, &dinit, &msg)) return fail(s, "%s", msg.c_str());
    DevBuf<double> col;
    CK(col.alloc((size_t)g.Ns * g.nc));
    k_entry_column_sum<<<g.Ns * g.nc, 256, 0, f->stream>>>(g, d_bar_gamma, col.p);
    CK(cudaGetLastError());
    std::vector<double> h((size_t)g.Ns * g.nc);
    CK(cudaMemcpyAsync(h.data(), col.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, f->stream));
    CK(cudaStreamSynchronize(f->stream));
    for (int q = 0; q < n_par; ++q) {
        double acc = 0.0;
        for (size_t e = 0; e < h.size(); ++e) acc += dinit[e * n_par + q] * h[e];
        grad[q] = acc;
    }
    return SR_OK;
}

// ----------------------------------------------------------------------------- batched flows
//
// Many flows (instances of uneven size) integrated together: every kernel of an Euler step
// covers all instances in one launch (blockIdx.y = instance for the small kernels); the
// vertex flow is one persistent kernel whose CTAs pull (instance, stored triple) units from
// an atomic counter, largest instances first.  The cutoff of step k is read on the device
// from a list, so one captured CUDA graph of the step replays the whole loop.

namespace {

struct BInst {
    Geo g;
    Tabs tb;
    TabsT tt;       // TRI tables (kind 3)
    double* gam;
    double* G;
    float* Gf;
    const float* Gs;
    double* dgam;
    double* dG;
    double* nx;
    double* nW;
    float* nWf;
    float* nxf;
    int* ncount;
    long unit0;     // first work unit (stored triple) of this instance
    int qc;         // integration nodes per shared-memory block
    int kind;       // 0 SU2 dense, 1 SU2 product list, 2 XYZ, 3 TRI
    int with_swap;
    int qb_own;     // SU2 dense: node block of the instance's own kernel (k_gamma_rhs_su2f)
};

__global__ void k_sigma_b(const BInst* __restrict__ I, const double* __restrict__ lams, const int* __restrict__ step) {
    const BInst& B = I[blockIdx.y];
    if ((int)blockIdx.x >= B.g.N) return;
    if (B.kind == 3) sigma_rhs_tri_block(B.g, B.tb, B.tt, B.tb.w, B.gam, B.G, lams[*step], B.dgam, blockIdx.x);
    else sigma_rhs_block<double>(B.g, B.tb, B.tb.w, B.gam, B.G, lams[*step], B.dgam, blockIdx.x);
}

__global__ void k_nodes_b(const BInst* __restrict__ I, const double* __restrict__ lams, const int* __restrict__ step) {
    const BInst& B = I[blockIdx.y];
    if ((int)blockIdx.x >= 3 * B.g.N) return;
    channel_nodes_block<double>(B.g, B.tb.w, B.tb.invh, B.gam, B.dgam, lams[*step], B.nx, B.nW, B.nWf, B.ncount, blockIdx.x,
                                B.nxf);
}

// One size class of instances: units [u_begin, u_end) (instances [i_begin, i_end)).
template <int NC, bool DENSE>
__global__ void __launch_bounds__(kThreads, 7) k_gamma_persistent(const BInst* __restrict__ I, int i_begin, int i_end,
                                                               long u_begin, long u_end,
                                                               unsigned long long* __restrict__ counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long unit_sh;
    __shared__ int inst_sh;
    __shared__ __align__(16) BInst B;   // the unit's instance, staged once per unit
    int cur = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const long u = u_begin + (long)atomicAdd(counter, 1ULL);
            int lo = i_begin, hi = i_end - 1;   // last instance with unit0 <= u
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (I[mid].unit0 <= u) lo = mid; else hi = mid - 1;
            }
            unit_sh = u;
            inst_sh = lo;
        }
        __syncthreads();
        const long u = unit_sh;
        if (u >= u_end) break;
        if (inst_sh != cur) {
            cur = inst_sh;
            static_assert(sizeof(BInst) % sizeof(int) == 0, "BInst copied as ints");
            const int* src = reinterpret_cast<const int*>(I + cur);
            for (int i = threadIdx.x; i < (int)(sizeof(BInst) / sizeof(int)); i += blockDim.x)
                reinterpret_cast<int*>(&B)[i] = src[i];
            __syncthreads();
        }
        const long local = u - B.unit0;
        const Geo g = B.g;   // locals: see k_gamma_persistent_su2f
        const Tabs tb = B.tb;
        const int p = (int)(local / g.N), ti = (int)(local % g.N);
        gamma_rhs_f32_triple<NC, DENSE>(g, tb, B.Gf, B.Gs, B.nxf, B.nWf, B.ncount, B.dG, p, ti, smem, B.qc);
    }
}

// SU2 instances (dense lattice sum) in one persistent kernel over the per-triple function of
// k_gamma_rhs_su2f: CTAs take `chunk` consecutive units per atomic step (consecutive units
// mostly belong to one instance, whose tables are staged once), with the register budget of
// the instances' own kernel.  CACHE: the corner-row cache of k_gamma_rhs_su2f<true> (classes of
// wide rows).
template <bool CACHE>
__global__ void __launch_bounds__(su2f::kThreadsS, CACHE ? su2f::kMinCtasCached : su2f::kMinCtas) k_gamma_persistent_su2f(const BInst* __restrict__ I, int i_begin, int i_end,
                                                                    long u_begin, long u_end,
                                                                    unsigned long long* __restrict__ counter, int chunk) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long unit_sh;
    __shared__ __align__(16) BInst B;   // the current unit's instance
    int cur = -1;
    long cur_end = -1;                  // first unit past the current instance
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) unit_sh = u_begin + (long)atomicAdd(counter, (unsigned long long)chunk);
        __syncthreads();
        const long u0 = unit_sh;
        if (u0 >= u_end) break;
        const long u1 = min(u0 + (long)chunk, u_end);
        for (long u = u0; u < u1; ++u) {
            if (cur < 0 || u < B.unit0 || u >= cur_end) {
                __shared__ int inst_sh;
                __syncthreads();
                if (threadIdx.x == 0) {
                    int lo = i_begin, hi = i_end - 1;   // last instance with unit0 <= u
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (I[mid].unit0 <= u) lo = mid; else hi = mid - 1;
                    }
                    inst_sh = lo;
                }
                __syncthreads();
                cur = inst_sh;
                static_assert(sizeof(BInst) % sizeof(int) == 0, "BInst copied as ints");
                const int* src = reinterpret_cast<const int*>(I + cur);
                for (int i = threadIdx.x; i < (int)(sizeof(BInst) / sizeof(int)); i += blockDim.x)
                    reinterpret_cast<int*>(&B)[i] = src[i];
                __syncthreads();
                cur_end = B.unit0 + (long)B.g.npair * B.g.N;
            }
            const long local = u - B.unit0;
            // the instance's geometry and tables as locals: the per-triple function's stores to
            // shared memory would otherwise force re-reads of every field from the shared copy
            const Geo g = B.g;
            const Tabs tb = B.tb;
            su2f::triple<CACHE>(g, tb, B.Gf, B.with_swap ? (int)g.nentp : 0, B.nxf, B.nWf, B.ncount, B.dG,
                                (int)(local / g.N), (int)(local % g.N), smem, B.qc);
        }
    }
}

// Units per atomic step of the SU2 persistent kernel.
constexpr int kUnitChunk = 4;

// Persistent kernel of an instance kind (0: SU2 dense lattice sum, 1: SU2 product list, 2: XYZ;
// TRI instances, kind 3, always run their own kernels); every size class holds instances of
// one kind.
static const void* persistent_fn(int kind, bool cache = false) {
    if (kind == 0) return cache ? (const void*)k_gamma_persistent_su2f<true> : (const void*)k_gamma_persistent_su2f<false>;
    if (kind == 1) return (const void*)k_gamma_persistent<2, false>;
    return (const void*)k_gamma_persistent<4, false>;
}

// Euler update of every instance (y <- y - (Lambda_k - Lambda_k+1) f) and its FP32 shadow.
__global__ void k_update_b(const BInst* __restrict__ I, const double* __restrict__ lams, const int* __restrict__ step,
                           int* __restrict__ flag) {
    const BInst& B = I[blockIdx.y];
    const double dl = lams[*step] - lams[*step + 1];
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < B.g.N; i += stride) {
        const double v = B.gam[i] - dl * B.dgam[i];
        if (!isfinite(v)) atomicOr(flag, 1);
        B.gam[i] = v;
    }
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < B.g.nent; i += stride) {
        const double v = B.G[i] - dl * B.dG[i];
        if (!isfinite(v)) atomicOr(flag, 1);
        B.G[i] = v;
    }
}

__global__ void k_shadow_b(const BInst* __restrict__ I) {
    const BInst& B = I[blockIdx.y];
    const Geo& g = B.g;
    const int rowp = g.nc * g.nsp;
    const long stride = (long)gridDim.x * blockDim.x;
    if (B.kind == 3) {
        // TRI: FP32 copy of the state in its own layout
        for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < g.nent; i += stride) B.Gf[i] = (float)B.G[i];
        return;
    }
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < g.nentp; i += stride) {
        const long pt = i / rowp;
        const int rem = (int)(i % rowp);
        const int c = rem / g.nsp, r = rem % g.nsp;
        const double* src = B.G + pt * g.nc * g.Ns;
        float v = 0.0f, vs = 0.0f;
        if (r < g.Ns) {
            v = (float)src[c * g.Ns + r];
            if (B.with_swap) vs = (float)src[perm_of(B.tb.swap_perm[r], c) * g.Ns + B.tb.swap_r[r]];
        }
        B.Gf[i] = v;
        if (B.with_swap) B.Gf[g.nentp + i] = vs;
    }
}

__global__ void k_advance(int* __restrict__ step, unsigned long long* __restrict__ counter, int ncounter) {
    *step += 1;
    for (int i = 0; i < ncounter; ++i) counter[i] = 0ULL;
}

}  // namespace

struct BClass {
    int kind;             // instance kind (persistent_fn)
    int i_begin, i_end;   // instances
    long u_begin, u_end;  // work units
    size_t smem;
    int occ, ctas, qc;
    int threads;          // CTA size of the class's persistent kernel
    bool cache;           // SU2: the corner-row cache (k_gamma_rhs_su2f<true>) for wide rows
    double ms;            // autotuned vertex-flow time of the class
    bool per_inst;        // the instances' own vertex kernels, one launch each, instead of the
                          // class's persistent kernel
};

struct sr_batch {
    std::vector<sr_flow*> flows;
    std::vector<BInst> inst;         // host copy, grouped in shared-memory classes, largest first
    std::vector<BClass> cls;
    DevBuf<BInst> dinst;
    DevBuf<double> lams;
    DevBuf<int> step;
    DevBuf<unsigned long long> counter;
    DevBuf<int> flag;
    cudaStream_t stream = nullptr;
    long total = 0;
    size_t smem = 0;
    int nsm = 0, occ = 1, ctas = 1, qc = kQF;
    double tune_ms = 0.0;
    double run_ms = 0.0;
    int n_lambda_cap = 0;
    std::vector<cudaStream_t> side;   // one per size class beyond the first
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    bool parallel = true;             // size classes as parallel branches (else one after another)
    int force = 0;                    // 0: the autotuner picks the launch form per class,
                                      // 1: persistent kernels, 2: per-instance kernels
    std::vector<size_t> inst_smem;    // per instance: dynamic shared memory of its own kernel
    ~sr_batch() {
        for (cudaStream_t s : side) cudaStreamDestroy(s);
        for (cudaEvent_t e : join) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (stream) cudaStreamDestroy(stream);
    }
};

static void launch_class(sr_batch* b, int k, cudaStream_t st) {
    const BClass& c = b->cls[k];
    if (c.per_inst || c.kind == 3) {
        // the instances' own vertex kernels (as a single flow launches them), back to back
        for (int i = c.i_begin; i < c.i_end; ++i) {
            const BInst& B = b->inst[i];
            const unsigned blocks = (unsigned)(B.g.npair * B.g.N);
            const size_t sm = b->inst_smem[i];
            if (c.kind == 0 && su2f::cache_for(B.g.nsp))
                k_gamma_rhs_su2f<true><<<blocks, su2f::threads_for(B.g.nsp), sm, st>>>(
                    B.g, B.tb, B.Gf, B.with_swap ? (int)B.g.nentp : 0, B.nxf, B.nWf, B.ncount, B.dG, B.qb_own, 0);
            else if (c.kind == 0)
                k_gamma_rhs_su2f<false><<<blocks, su2f::threads_for(B.g.nsp), sm, st>>>(
                    B.g, B.tb, B.Gf, B.with_swap ? (int)B.g.nentp : 0, B.nxf, B.nWf, B.ncount, B.dG, B.qb_own, 0);
            else if (c.kind == 1)
                k_gamma_rhs_f32<2, false><<<blocks, kThreads, sm, st>>>(B.g, B.tb, B.Gf, B.Gs, B.nxf, B.nWf, B.ncount, B.dG, 0);
            else if (c.kind == 3)
                k_gamma_rhs_tri<float><<<blocks, kThreads, sm, st>>>(B.g, B.tb, B.tt, B.tb.w, B.Gf, B.nx, B.nW, B.ncount, B.dG, 0);
            else
                k_gamma_rhs_f32<4, false><<<blocks, kThreads, sm, st>>>(B.g, B.tb, B.Gf, B.Gs, B.nxf, B.nWf, B.ncount, B.dG, 0);
        }
        return;
    }
    const dim3 grid(b->nsm * c.ctas);
    unsigned long long* ctr = b->counter.p + k;
    if (c.kind == 0)
        (c.cache ? k_gamma_persistent_su2f<true> : k_gamma_persistent_su2f<false>)<<<grid, c.threads, c.smem, st>>>(
            b->dinst.p, c.i_begin, c.i_end, c.u_begin, c.u_end, ctr, kUnitChunk);
    else if (c.kind == 1)
        k_gamma_persistent<2, false><<<grid, kThreads, c.smem, st>>>(b->dinst.p, c.i_begin, c.i_end, c.u_begin, c.u_end, ctr);
    else
        k_gamma_persistent<4, false><<<grid, kThreads, c.smem, st>>>(b->dinst.p, c.i_begin, c.i_end, c.u_begin, c.u_end, ctr);
}

// The vertex flow of every size class: as parallel branches (fork / join, so a class's tail
// overlaps the others) or one after another on the batch stream, as the autotuner chose.
static sr_status launch_classes(sr_batch* b) {
    const int nk = (int)b->cls.size();
    if (b->parallel && nk > 1) {
        CK(cudaEventRecord(b->fork, b->stream));
        for (int k = 1; k < nk; ++k) {
            CK(cudaStreamWaitEvent(b->side[k - 1], b->fork, 0));
            launch_class(b, k, b->side[k - 1]);
            CK(cudaEventRecord(b->join[k - 1], b->side[k - 1]));
        }
        launch_class(b, 0, b->stream);
        for (int k = 1; k < nk; ++k) CK(cudaStreamWaitEvent(b->stream, b->join[k - 1], 0));
    } else {
        for (int k = 0; k < nk; ++k) launch_class(b, k, b->stream);
    }
    return SR_OK;
}

static sr_status batch_launch_step(sr_batch* b) {
    const int ni = (int)b->inst.size();
    int maxN = 0;
    long maxent = 0;
    for (const BInst& B : b->inst) { maxN = std::max(maxN, B.g.N); maxent = std::max(maxent, B.g.nentp); }
    k_sigma_b<<<dim3(maxN, ni), 64, 0, b->stream>>>(b->dinst.p, b->lams.p, b->step.p);
    k_nodes_b<<<dim3(3 * maxN, ni), 128, 0, b->stream>>>(b->dinst.p, b->lams.p, b->step.p);
    if (sr_status s = launch_classes(b)) return s;
    const int ub = (int)std::min<long>((maxent + 255) / 256, 4 * b->nsm);
    k_update_b<<<dim3(ub, ni), 256, 0, b->stream>>>(b->dinst.p, b->lams.p, b->step.p, b->flag.p);
    k_shadow_b<<<dim3(ub, ni), 256, 0, b->stream>>>(b->dinst.p);
    k_advance<<<1, 1, 0, b->stream>>>(b->step.p, b->counter.p, (int)b->cls.size());
    CK(cudaGetLastError());
    return SR_OK;
}

static sr_status batch_upload(sr_batch* b) {
    CK(cudaMemcpyAsync(b->dinst.p, b->inst.data(), sizeof(BInst) * b->inst.size(), cudaMemcpyHostToDevice, b->stream));
    return SR_OK;
}

// Time the vertex flow of one size class (its persistent kernel alone).
static sr_status batch_time_class(sr_batch* b, int k, double* ms) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
        CK(cudaMemsetAsync(b->counter.p + k, 0, sizeof(unsigned long long), b->stream));
        CK(cudaEventRecord(e0, b->stream));
        launch_class(b, k, b->stream);
        CK(cudaGetLastError());
        CK(cudaEventRecord(e1, b->stream));
        CK(cudaEventSynchronize(e1));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        best = std::min(best, t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return SR_OK;
}

// Autotuner: per size class, the node-block size and the CTAs per SM of its persistent
// kernel, each candidate timed on the current state and node tables, against the instances'
// own kernels launched one after another; the fastest is kept.
static sr_status batch_tune(sr_batch* b) {
    const int qcs[3] = {8, 16, 32};
    double total = 0.0;
    for (int k = 0; k < (int)b->cls.size(); ++k) {
        BClass& c = b->cls[k];
        c.per_inst = false;
        if (b->force == 2 || c.kind == 3) {
            c.per_inst = true;
            double ms = 0;
            if (sr_status s = batch_time_class(b, k, &ms)) return s;
            c.ms = ms;
            total += ms;
            continue;
        }
        // candidates (node block, shared memory, resident CTAs per SM): SU2 launches with the
        // shared memory its node block needs, so small blocks raise the occupancy
        struct Cand { int qc; size_t smem; int occ; };
        std::vector<Cand> cand;
        if (c.kind == 0) {
            for (int qb : {16, 32, 64}) {
                size_t need = 0;
                for (int i = c.i_begin; i < c.i_end; ++i)
                    need = std::max(need, su2f::layout(b->inst[i].g.N, b->inst[i].g.Ns, b->inst[i].g.nsp, qb, c.threads).total);
                if (need > 227 * 1024) continue;
                CK(ensure_smem(persistent_fn(c.kind, c.cache), need));
                int occ = 0;
                CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persistent_fn(c.kind, c.cache), c.threads, need));
                if (occ >= 1) cand.push_back({qb, need, occ});
            }
        } else {
            for (int qb : qcs) cand.push_back({qb, c.smem, c.occ});
        }
        if (cand.empty()) return fail(SR_EUNSUPPORTED, "size class %d: no node block fits the persistent kernel", k);
        double best = 1e300;
        int bq = c.qc, bc = c.ctas;
        size_t bs = c.smem;
        for (const Cand& q : cand)
            for (int ct = q.occ; ct >= 1; ct = ct > 2 ? ct - (ct + 3) / 4 : ct - 1) {
                for (int i = c.i_begin; i < c.i_end; ++i) b->inst[i].qc = q.qc;
                c.ctas = ct;
                c.smem = q.smem;
                if (sr_status s = batch_upload(b)) return s;
                double ms = 0;
                if (sr_status s = batch_time_class(b, k, &ms)) return s;
                if (ms < best) { best = ms; bq = q.qc; bc = ct; bs = q.smem; }
                if (ct <= q.occ / 2) break;   // fewer CTAs than half the occupancy: not worth timing
            }
        for (int i = c.i_begin; i < c.i_end; ++i) b->inst[i].qc = bq;
        c.ctas = bc;
        c.qc = bq;
        c.smem = bs;
        c.ms = best;
        if (b->force == 0) {
            c.per_inst = true;
            double ms = 0;
            if (sr_status s = batch_time_class(b, k, &ms)) return s;
            if (ms < best) c.ms = ms;
            else c.per_inst = false;
        }
        total += c.ms;
    }
    b->tune_ms = total;
    b->qc = b->cls.empty() ? kQF : b->cls[0].qc;
    b->ctas = b->cls.empty() ? 1 : b->cls[0].ctas;
    if (sr_status s = batch_upload(b)) return s;
    // then the classes together: parallel branches or one after another, for the per-class
    // choices and (unless a form is forced) for every class persistent and every class on its
    // instances' own kernels, since classes timed alone miss how their tails overlap; the
    // fastest combination is kept
    if (b->cls.size() > 1) {
        const int nk = (int)b->cls.size();
        std::vector<std::vector<bool>> forms;
        std::vector<bool> tuned(nk);
        for (int k = 0; k < nk; ++k) tuned[k] = b->cls[k].per_inst;
        forms.push_back(tuned);
        if (b->force == 0) {
            std::vector<bool> pers(nk), own(nk, true);
            for (int k = 0; k < nk; ++k) pers[k] = b->cls[k].kind == 3;
            forms.push_back(pers);
            forms.push_back(own);
        }
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        double best = 1e300;
        size_t best_form = 0;
        bool best_par = false;
        for (size_t fi = 0; fi < forms.size(); ++fi) {
            for (int k = 0; k < nk; ++k) b->cls[k].per_inst = forms[fi][k];
            for (int rep = 0; rep < 2; ++rep)
                for (int mode = 0; mode < 2; ++mode) {
                    b->parallel = mode == 1;
                    CK(cudaMemsetAsync(b->counter.p, 0, sizeof(unsigned long long) * b->cls.size(), b->stream));
                    CK(cudaEventRecord(e0, b->stream));
                    if (sr_status s = launch_classes(b)) return s;
                    CK(cudaEventRecord(e1, b->stream));
                    CK(cudaEventSynchronize(e1));
                    float t = 0.f;
                    CK(cudaEventElapsedTime(&t, e0, e1));
                    if (t < best) { best = t; best_form = fi; best_par = mode == 1; }
                }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (int k = 0; k < nk; ++k) b->cls[k].per_inst = forms[best_form][k];
        b->parallel = best_par;
        b->tune_ms = best;
    }
    return SR_OK;
}

extern "C" sr_status sr_batch_parallel_classes(const sr_batch* b, int* parallel) {
    if (!b || !parallel) return fail(SR_EINVAL, "null argument");
    *parallel = b->parallel ? 1 : 0;
    return SR_OK;
}

extern "C" sr_status sr_batch_create(int n, sr_flow* const* flows, sr_batch** out) {
    if (n <= 0 || !flows || !out) return fail(SR_EINVAL, "need at least one flow");
    *out = nullptr;
    std::unique_ptr<sr_batch> b(new (std::nothrow) sr_batch());
    if (!b) return fail(SR_ENOMEM, "out of host memory");
    for (int i = 0; i < n; ++i) {
        sr_flow* f = flows[i];
        if (!f) return fail(SR_EINVAL, "null flow %d", i);
        if (f->prec != SR_FP32_MIXED) return fail(SR_EUNSUPPORTED, "batched flows use the FP32-mixed kernels (flow %d is FP64)", i);
        b->flows.push_back(f);
    }
    // instances grouped by kind and by the shared memory their vertex flow needs (each class
    // gets a persistent launch sized for it), largest first; within a class, largest instance
    // first
    std::vector<size_t> sm(n);
    std::vector<int> kind(n);
    for (int i = 0; i < n; ++i) {
        sr_flow* f = flows[i];
        kind[i] = f->g.nc == 16 ? 3 : (f->g.nc == 4 ? 2 : (f->dense ? 0 : 1));
        if (kind[i] == 0 && f->su2f_qb == 0)
            return fail(SR_EUNSUPPORTED, "flow %d: lattice too large for the batched SU2 kernel", i);
        // SU2 dense: shared memory of the largest node block that fits (the tuner may pick it)
        if (kind[i] == 0) {
            const int nth = su2f::threads_for(f->g.nsp);
            sm[i] = f->smem_su2f;
            for (int qb : {64, 32}) {
                const size_t bq = su2f::layout(f->g.N, f->g.Ns, f->g.nsp, qb, nth).total;
                if (bq <= 227 * 1024 / 3) { sm[i] = std::max(sm[i], bq); break; }
            }
        } else if (kind[i] == 3) {
            sm[i] = f->smem_rhs;
        } else {
            sm[i] = f32_smem_bytes(f->g.Ns, f->g.nsp, f->g.nc, f->nprod, f->dense);
        }
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    // SU2 instances whose own kernel is k_gamma_rhs_su2f<true> (wide rows) form classes of their
    // own, so that every class's persistent kernel has its instances' CTA size and variant
    auto wide = [&](int i) { return kind[i] == 0 && su2f::cache_for(flows[i]->g.nsp); };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        if (kind[a] != kind[c]) return kind[a] < kind[c];
        if (wide(a) != wide(c)) return wide(a);
        if (sm[a] != sm[c]) return sm[a] > sm[c];
        return flows[a]->g.nent > flows[c]->g.nent;
    });
    long unit = 0;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev));
    for (int idx = 0; idx < n; ++idx) {
        const int k = order[idx];
        sr_flow* f = flows[k];
        // a new class for a new kind or row width, or when the shared memory drops below 2/3 of
        // the class's largest
        if (b->cls.empty() || b->cls.back().kind != kind[k] || b->cls.back().cache != wide(k) ||
            sm[k] * 3 < b->cls.back().smem * 2) {
            BClass c{};
            c.kind = kind[k];
            c.i_begin = idx; c.u_begin = unit; c.smem = sm[k]; c.qc = kind[k] == 0 ? f->su2f_qb : kQF;
            c.threads = kind[k] == 0 ? su2f::threads_for(f->g.nsp) : kThreads;
            c.cache = kind[k] == 0 && su2f::cache_for(f->g.nsp);
            if (sm[k] > 227 * 1024) return fail(SR_EUNSUPPORTED, "instance needs %zu bytes of shared memory", sm[k]);
            if (c.kind == 3) {
                c.occ = 1;   // no persistent kernel: the instances' own launches
                c.per_inst = true;
            } else {
                CK(ensure_smem(persistent_fn(c.kind, c.cache), sm[k]));
                CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ, persistent_fn(c.kind, c.cache), c.threads, sm[k]));
                if (c.occ < 1) return fail(SR_EUNSUPPORTED, "persistent kernel cannot be resident with %zu bytes", sm[k]);
            }
            c.ctas = c.occ;
            b->cls.push_back(c);
        }
        BInst B;
        B.g = f->g;
        B.tb = f->tabs();
        B.tt = kind[k] == 3 ? f->tabs_tri() : TabsT{};
        B.gam = f->gam.p; B.G = f->G.p; B.Gf = f->Gf.p; B.Gs = f->has_swap ? f->Gf.p + f->g.nentp : f->Gf.p;
        B.dgam = f->dgam.p; B.dG = f->dG.p; B.nx = f->nx.p; B.nW = f->nW.p; B.nWf = f->nWf.p; B.nxf = f->nxf.p;
        B.ncount = f->ncount.p;
        B.unit0 = unit;
        B.qc = kQF;
        B.kind = kind[k];
        B.with_swap = f->has_swap ? 1 : 0;
        B.qb_own = f->su2f_qb;
        if (kind[k] == 0) B.qc = f->su2f_qb;
        unit += (long)f->g.npair * f->g.N;
        b->inst.push_back(B);
        b->inst_smem.push_back(kind[k] == 0 ? f->smem_su2f : f->smem_rhs);   // TRI: k_gamma_rhs_tri<float>
        b->cls.back().i_end = idx + 1;
        b->cls.back().u_end = unit;
    }
    b->total = unit;
    b->smem = b->cls.front().smem;
    b->occ = b->cls.front().occ;
    b->ctas = b->occ;
    CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    for (size_t k = 1; k < b->cls.size(); ++k) {
        cudaStream_t st;
        cudaEvent_t ev;
        CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        b->side.push_back(st);
        b->join.push_back(ev);
    }
    CK(b->dinst.alloc(b->inst.size()));
    CK(b->step.alloc(1));
    CK(b->counter.alloc(b->cls.size()));
    CK(cudaMemsetAsync(b->counter.p, 0, sizeof(unsigned long long) * b->cls.size(), b->stream));
    CK(b->flag.alloc(1));
    if (sr_status s = batch_upload(b.get())) return s;
    CK(cudaStreamSynchronize(b->stream));
    *out = b.release();
    return SR_OK;
}

extern "C" sr_status sr_batch_run(sr_batch* b, int n_lambda, const double* lambdas, int use_graph, int autotune) {
    if (!b || n_lambda < 2 || !lambdas) return fail(SR_EINVAL, "need a batch and at least two cutoffs");
    for (int i = 0; i + 1 < n_lambda; ++i)
        if (!(lambdas[i + 1] < lambdas[i]) || !(lambdas[i + 1] > 0.0)) return fail(SR_EINVAL, "cutoffs must decrease and stay positive");
    for (sr_flow* f : b->flows) {
        if (std::fabs(f->lambda - lambdas[0]) > 1e-12 * lambdas[0]) return fail(SR_EINVAL, "every flow must start at lambdas[0]");
        CK(cudaStreamSynchronize(f->stream));
    }
    if (b->n_lambda_cap < n_lambda) { CK(b->lams.alloc(n_lambda)); b->n_lambda_cap = n_lambda; }
    CK(cudaMemcpyAsync(b->lams.p, lambdas, sizeof(double) * n_lambda, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemsetAsync(b->step.p, 0, sizeof(int), b->stream));
    CK(cudaMemsetAsync(b->counter.p, 0, sizeof(unsigned long long) * b->cls.size(), b->stream));
    CK(cudaMemsetAsync(b->flag.p, 0, sizeof(int), b->stream));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int nsteps = n_lambda - 1;
    int done = 0;
    if (autotune) {
        // tune on node tables at the middle cutoff of the run (self-energy flow and nodes of
        // the current state at that cutoff): the integration nodes, and with them the work per
        // stored triple, grow as the cutoff falls, and the launch forms' ranking with them, so
        // the first step's tables under-represent the run
        const int ni = (int)b->inst.size();
        int maxN = 0;
        for (const BInst& B : b->inst) maxN = std::max(maxN, B.g.N);
        const int mid = nsteps / 2;
        CK(cudaMemcpyAsync(b->step.p, &mid, sizeof(int), cudaMemcpyHostToDevice, b->stream));
        k_sigma_b<<<dim3(maxN, ni), 64, 0, b->stream>>>(b->dinst.p, b->lams.p, b->step.p);
        k_nodes_b<<<dim3(3 * maxN, ni), 128, 0, b->stream>>>(b->dinst.p, b->lams.p, b->step.p);
        CK(cudaGetLastError());
        if (sr_status s = batch_tune(b)) return s;
        // back to the first step, with the work counters the tuning launches consumed reset
        // (a persistent kernel started on a spent counter would skip the first step's units)
        CK(cudaMemsetAsync(b->step.p, 0, sizeof(int), b->stream));
        CK(cudaMemsetAsync(b->counter.p, 0, sizeof(unsigned long long) * b->cls.size(), b->stream));
    }
    if (use_graph) {
        cudaGraph_t graph;
        cudaGraphExec_t exec;
        CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        sr_status s = batch_launch_step(b);
        cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
        if (s != SR_OK) return s;
        if (ce != cudaSuccess) return fail(SR_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
        CK(cudaGraphInstantiate(&exec, graph, 0));
        CK(cudaGraphUpload(exec, b->stream));
        CK(cudaEventRecord(e0, b->stream));   // run time: the replays, not the capture
        for (; done < nsteps; ++done) CK(cudaGraphLaunch(exec, b->stream));
        CK(cudaStreamSynchronize(b->stream));
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
    } else {
        CK(cudaEventRecord(e0, b->stream));
        for (; done < nsteps; ++done)
            if (sr_status s = batch_launch_step(b)) return s;
    }
    CK(cudaEventRecord(e1, b->stream));
    CK(cudaEventSynchronize(e1));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, e0, e1));
    b->run_ms = t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int fl = 0;
    CK(cudaMemcpy(&fl, b->flag.p, sizeof(int), cudaMemcpyDeviceToHost));
    for (sr_flow* f : b->flows) {
        f->lambda = lambdas[n_lambda - 1];
        f->fsal = false;
        f->n_rhs += nsteps;
    }
    if (fl) return fail(SR_ENONFINITE, "non-finite value in a batched flow");
    return SR_OK;
}

extern "C" sr_status sr_batch_info(const sr_batch* b, int* qc, int* ctas_per_sm, double* tune_ms, double* run_ms,
                                   long* units) {
    if (!b) return fail(SR_EINVAL, "null batch");
    if (qc) *qc = b->qc;
    if (ctas_per_sm) *ctas_per_sm = b->ctas;
    if (tune_ms) *tune_ms = b->tune_ms;
    if (run_ms) *run_ms = b->run_ms;
    if (units) *units = b->total;
    return SR_OK;
}

extern "C" sr_status sr_batch_force_launch(sr_batch* b, int mode) {
    if (!b || mode < 0 || mode > 2) return fail(SR_EINVAL, "mode must be 0 (autotune), 1 (persistent) or 2 (per instance)");
    b->force = mode;
    if (mode != 0)
        for (BClass& c : b->cls) c.per_inst = mode == 2 || c.kind == 3;
    return SR_OK;
}

extern "C" sr_status sr_batch_class_launch(const sr_batch* b, int k, int* per_instance) {
    if (!b || !per_instance || k < 0 || k >= (int)b->cls.size()) return fail(SR_EINVAL, "bad class index");
    *per_instance = b->cls[k].per_inst ? 1 : 0;
    return SR_OK;
}

extern "C" sr_status sr_batch_classes(const sr_batch* b, int* n_classes) {
    if (!b || !n_classes) return fail(SR_EINVAL, "null argument");
    *n_classes = (int)b->cls.size();
    return SR_OK;
}

extern "C" sr_status sr_batch_class(const sr_batch* b, int k, int* n_instances, long* units, int* smem_bytes, int* qc,
                                    int* ctas_per_sm, double* tune_ms) {
    if (!b || k < 0 || k >= (int)b->cls.size()) return fail(SR_EINVAL, "bad class index");
    const BClass& c = b->cls[k];
    if (n_instances) *n_instances = c.i_end - c.i_begin;
    if (units) *units = c.u_end - c.u_begin;
    if (smem_bytes) *smem_bytes = (int)c.smem;
    if (qc) *qc = c.qc;
    if (ctas_per_sm) *ctas_per_sm = c.ctas;
    if (tune_ms) *tune_ms = c.ms;
    return SR_OK;
}

extern "C" sr_status sr_batch_destroy(sr_batch* b) {
    if (b && b->stream) cudaStreamSynchronize(b->stream);
    delete b;
    return SR_OK;
}

// ----------------------------------------------------------------------------- allocation-free chi(k)

// Scratch of the allocation-free correlation measurement: the chi_ij pair table.  Device
// code could name it directly; host code must not pass the symbol itself (it is a
// host-side stand-in), so its device address is looked up once per device.
static __device__ __align__(256) double g_chi_static[SR_CHI_STATIC_MAX];
static std::mutex g_chi_static_mu;
static double* g_chi_static_ptr[64] = {nullptr};

extern "C" sr_status sr_measure_susceptibility_static(sr_flow* f, int n_k, const double* d_k_xyz, double* d_chi_k) {
    if (!f) return fail(SR_EINVAL, "null flow");
    if (f->ntan) return fail(SR_EINVAL, "tangent flows measure with sr_measure_susceptibility_tangent");
    if (n_k < 0 || (n_k > 0 && (!d_k_xyz || !d_chi_k))) return fail(SR_EINVAL, "bad momenta or output");
    const sr_lattice* lat = f->lat;
    const Geo& g = f->g;
    const int npairs = (int)lat->chi_map.size();
    const size_t need = (size_t)npairs * g.nc;
    if (need > (size_t)SR_CHI_STATIC_MAX)
        return fail(SR_EINVAL, "correlation table needs %zu values, above the static limit of %d", need, SR_CHI_STATIC_MAX);
    // the array's address is per device: look it up (and launch) with the flow's device current
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev != f->device)
        return fail(SR_EINVAL, "device %d is current, but the flow lives on device %d: make the flow's device current", dev,
                    f->device);
    if (dev < 0 || dev >= 64) return fail(SR_EINVAL, "device index %d out of range", dev);
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_chi_static_mu);
        if (!g_chi_static_ptr[dev]) {
            void* p = nullptr;
            CK(cudaGetSymbolAddress(&p, g_chi_static));
            g_chi_static_ptr[dev] = (double*)p;
        }
        scratch = g_chi_static_ptr[dev];
    }
    Tabs tb = f->tabs();
    if (g.nc == 16)
        k_chi_tri<<<npairs, 128, 0, f->stream>>>(g, tb, f->tabs_tri(), f->w.p, f->gam.p, f->G.p, f->lambda, f->chi_r16.p, f->chi_m16.p,
                                                 f->chi_onsite.p, lat->Ntot, scratch);
    else if (g.nc == 2)
        k_chi<double, 2><<<npairs, 128, 0, f->stream>>>(g, tb, f->w.p, f->gam.p, f->G.p, f->lambda, f->chi_map.p, f->chi_onsite.p, lat->Ntot, scratch);
    else
        k_chi<double, 4><<<npairs, 128, 0, f->stream>>>(g, tb, f->w.p, f->gam.p, f->G.p, f->lambda, f->chi_map.p, f->chi_onsite.p, lat->Ntot, scratch);
    CK(cudaGetLastError());
    if (n_k > 0) {
        if (g.nc == 16)
            k_chi_k_tri<<<(n_k + 127) / 128, 128, 0, f->stream>>>(n_k, d_k_xyz, scratch, f->chi_dr.p, npairs, lat->nb, d_chi_k);
        else
            k_chi_k<double><<<(n_k + 127) / 128, 128, 0, f->stream>>>(n_k, d_k_xyz, scratch, f->chi_dr.p, npairs, lat->nb, g.nc, d_chi_k);
        CK(cudaGetLastError());
    }
    return SR_OK;
}

extern "C" sr_status sr_flow_chi_sites(const sr_flow* f, int* sites) {
    if (!f || !sites) return fail(SR_EINVAL, "null argument");
    const auto& cs = f->lat->chi_sites;
    for (size_t i = 0; i < cs.size(); ++i) {
        sites[4 * i] = cs[i].n[0]; sites[4 * i + 1] = cs[i].n[1]; sites[4 * i + 2] = cs[i].n[2]; sites[4 * i + 3] = cs[i].b;
    }
    return SR_OK;
}

extern "C" sr_status sr_flow_get_state(const sr_flow* f, double* d_sigma, double* d_gamma) {
    if (!f) return fail(SR_EINVAL, "null flow");
    if (d_sigma) CK(cudaMemcpyAsync(d_sigma, f->gam.p, sizeof(double) * f->g.N * f->ts, cudaMemcpyDeviceToDevice, f->stream));
    if (d_gamma) CK(cudaMemcpyAsync(d_gamma, f->G.p, sizeof(double) * f->g.nent * f->ts, cudaMemcpyDeviceToDevice, f->stream));
    return SR_OK;
}

extern "C" sr_status sr_flow_set_state(sr_flow* f, double lambda, const double* d_sigma, const double* d_gamma) {
    if (!f) return fail(SR_EINVAL, "null flow");
    if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(SR_EINVAL, "lambda must be positive");
    if (d_sigma) CK(cudaMemcpyAsync(f->gam.p, d_sigma, sizeof(double) * f->g.N * f->ts, cudaMemcpyDeviceToDevice, f->stream));
    if (d_gamma) CK(cudaMemcpyAsync(f->G.p, d_gamma, sizeof(double) * f->g.nent * f->ts, cudaMemcpyDeviceToDevice, f->stream));
    if (sr_status s = refresh_shadow(f, f->G.p, f->Gf.p)) return s;
    f->lambda = lambda;
    f->h_next = 0.0;
    f->err_prev = 1e-4;
    f->fsal = false;
    return SR_OK;
}

extern "C" sr_status sr_flow_lambda(const sr_flow* f, double* lambda) {
    if (!f || !lambda) return fail(SR_EINVAL, "null argument");
    *lambda = f->lambda;
    return SR_OK;
}

static void clear_profile(sr_flow* f) {
    for (int k = 0; k < 3; ++k) {
        for (auto& pr : f->ev[k]) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
        f->ev[k].clear();
    }
}

extern "C" sr_status sr_flow_destroy(sr_flow* f) {
    if (f && f->stream) cudaStreamSynchronize(f->stream);
    if (f) clear_profile(f);
    delete f;
    return SR_OK;
}

extern "C" sr_status sr_flow_profile_enable(sr_flow* f, int on) {
    if (!f) return fail(SR_EINVAL, "null flow");
    CK(cudaStreamSynchronize(f->stream));
    clear_profile(f);
    f->profiling = on != 0;
    return SR_OK;
}

extern "C" sr_status sr_flow_profile_read(sr_flow* f, double* ms, long* launches) {
    if (!f || !ms || !launches) return fail(SR_EINVAL, "null argument");
    CK(cudaStreamSynchronize(f->stream));
    for (int k = 0; k < 3; ++k) {
        double acc = 0.0;
        for (auto& pr : f->ev[k]) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, pr.first, pr.second));
            acc += t;
        }
        ms[k] = acc;
        launches[k] = (long)f->ev[k].size();
    }
    return SR_OK;
}

extern "C" sr_status sr_flow_launch_info(const sr_flow* f, int* info) {
    if (!f || !info) return fail(SR_EINVAL, "null argument");
    info[0] = f->tc_grid;
    info[1] = (int)f->smem_tc;
    info[2] = f->tc_occ_api;
    info[3] = (int)f->smem_rhs;
    return SR_OK;
}

extern "C" sr_status sr_flow_lattice_sum_products(const sr_flow* f, long* n) {
    if (!f || !n) return fail(SR_EINVAL, "null argument");
    *n = f->nprod;
    return SR_OK;
}

extern "C" sr_status sr_flow_node_counts(const sr_flow* f, int* counts) {
    if (!f || !counts) return fail(SR_EINVAL, "null argument");
    CK(cudaMemcpyAsync(counts, f->ncount.p, sizeof(int) * 3 * f->g.N, cudaMemcpyDeviceToHost, f->stream));
    CK(cudaStreamSynchronize(f->stream));
    return SR_OK;
}

namespace {
template <typename T>
__global__ void k_fma_peak(T* out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)-1.2345) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" sr_status sr_peak_fma(int precision, double* flops) {
    if (!flops) return fail(SR_EINVAL, "null argument");
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = nsm * 8;
    const int iters = precision == SR_FP64 ? 4096 : 65536;
    void* buf = nullptr;
    CK(cudaMalloc(&buf, sizeof(double) * threads * blocks));
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        CK(cudaEventRecord(a));
        if (precision == SR_FP64) k_fma_peak<double><<<blocks, threads>>>((double*)buf, iters, 0.999999, 1e-7);
        else k_fma_peak<float><<<blocks, threads>>>((float*)buf, iters, 0.999999f, 1e-7f);
        CK(cudaEventRecord(b));
        CK(cudaEventSynchronize(b));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, a, b));
        if (rep > 0) best = std::min(best, t);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    *flops = 2.0 * 8.0 * (double)iters * threads * blocks / (best * 1e-3);
    return SR_OK;
}
