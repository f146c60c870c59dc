// Kernels of the TRI core: the flow of all 16 basis functions Gamma^{mu nu} (FP64 state; the
// lookups and vertex products in FP64, or in FP32 for the mixed-precision flow).
//
// Included by flow.cu after the forward kernels, whose propagators, node arguments and lookup
// descriptors it shares.  Equations: arXiv:2109.13317, Sec. 3 (Eqs. frg:flowexplicit:1particle
// and frg:flowexplicit:2particle with the parametrization Eq. frg:parametrization and the
// relations Eq. frg:parametrizationBasis2p), discretised as in Sec. 4.2.  Storage: real
// g^{mu nu} with Gamma^{mu nu} = i^{iota} g^{mu nu} (tri_coef.h), layout
// [pair(s,u)][t][mu * 4 + nu][site] like the SU2 and XYZ cores.
//
// Lookup: the descriptor of make_desc folds the frequencies (t -> -t, s -> -s and u -> -u
// with site exchange, s <-> u) and keeps two corner-weight sets, for functions whose second
// spin index is 0 (factor -1 under s <-> u) and for the others; the TRI core adds the sign
// xi(mu) xi(nu) of t -> -t and u -> -u for the six imaginary-class functions (`mneg`), and
// the site exchange reads component nu mu of the exchanged pair (folded into swap_map).
#pragma once

#include "tri_coef.h"

namespace {

constexpr int kQTri = 8;   // integration nodes per shared-memory block of the TRI kernel

struct TabsT {
    const int* swap_map;    // 16 * Ns, component-major ([c * Ns + r]): component map of the
                            // exchanged pair (transposed)
    const int* onsite_map;  // Ns * 16: component map of (rep, rep) onto site 0
    const uint4* lat_rec;   // P * 4: per lattice-sum table entry, 32 16-bit codes: the row slot
                            // (tri_slot(rA, stored component)) of A^{mu l} (codes 0..15, mu * 4 + l)
                            // and the row slot of B^{l nu} (codes 16..31); bit 15 of codes 0..11
                            // carries the factorised signs (tri_lattice_item)
    const int4* lat_items;  // n_items: (site r, first entry, end entry, 0), the entries of r split
                            // into chunks; items of a site are consecutive
    const int* lat_item_off;  // Ns + 1: items of each site
    int n_items;
    const int* lat_off;     // Ns * 16 + 1: per output (site, component) its signed products
    const int2* lat_ent;    // (row-A slot, row-B slot or its complement for a negative sign)
};

__device__ __forceinline__ bool tri_mixed(int c) { return ((c >> 2) == 0) != ((c & 3) == 0); }

// Value type of a lookup with weights W in a state of type S: W, or the dual number of a
// tangent flow's state.
template <typename W, typename S> struct TriVal { using type = W; };
template <typename W, int P> struct TriVal<W, Dual<P>> { using type = Dual<P>; };

// Component c of the pair (ref, rep_r) at the descriptor's frequencies, interpolated in the
// descriptor's weight type W (FP64, or FP32 in the mixed-precision vertex kernel; dual
// numbers for a tangent flow's state).
template <typename W, typename S>
__device__ __forceinline__ typename TriVal<W, S>::type tri_value(const S* __restrict__ G, const Desc<W>& d, bool mneg,
                                                                 const Tabs& tb, const TabsT& tt, const Geo& g, int r, int c) {
    using V = typename TriVal<W, S>::type;
    int rs = r, m = c;
    if (d.swap) { rs = tb.swap_r[r]; m = tt.swap_map[c * g.Ns + r]; }
    const int cs = m & 15;
    const S* base = G + cs * g.Ns + rs;
    const W* wgt = (cs & 3) == 0 ? d.wd : d.ws;
    V acc = V(0);
    for (int k = 0; k < d.n; ++k) acc = fmadd((V)base[d.off[k]], wgt[k], acc);
    const bool neg = ((m & 16) != 0) != (mneg && tri_mixed(c));
    return neg ? -acc : acc;
}

// Self-energy flow (spin trace): dgamma(w) = -(1/2pi) sum_{w2 = +-Lambda} H / (w2 + gamma(w2)),
// H = 2 sum_j Gamma^00_{ref j}(w+w2, 0, w-w2) - sum_k Gamma^kk_{ref ref}(w+w2, w2-w, 0).
// (block n: the frequency w[n]; any block size up to 1024 threads; T: double, or the dual
// numbers of a tangent flow)
template <typename T>
__device__ void sigma_rhs_tri_block(const Geo& g, const Tabs& tb, const TabsT& tt, const double* __restrict__ w,
                                    const T* __restrict__ gam, const T* __restrict__ G, double lam,
                                    T* __restrict__ dgam, int n) {
    __shared__ double red[2 * 32 * (sizeof(T) / sizeof(double))];
    const double w1 = w[n];
    T H[2] = {T(0.0), T(0.0)};
    for (int sg = 0; sg < 2; ++sg) {
        const double w2 = sg == 0 ? lam : -lam;
        Desc<double> d;
        make_desc(w1 + w2, 0.0, w1 - w2, 1, 0, tb, g, d);
        const bool mn = (w1 - w2) < 0.0;
        T h = T(0.0);
        for (int r = threadIdx.x; r < g.Ns; r += blockDim.x) h += (double)tb.mult[r] * tri_value(G, d, mn, tb, tt, g, r, 0);
        h = 2.0 * h;
        if (threadIdx.x == 0) {
            Desc<double> e;
            make_desc(w1 + w2, w2 - w1, 0.0, 2, 0, tb, g, e);
            const bool me = (w2 - w1) < 0.0;
            T f = T(0.0);
            for (int k = 0; k < 4; ++k) f += tri_value(G, e, me, tb, tt, g, 0, 5 * k);
            h -= f;
        }
        H[sg] = h;
    }
    block_sum<T, 2>(H, red);
    if (threadIdx.x == 0) {
        T acc = H[0] / (lam + interp_odd(w, tb.invh, g.N, gam, lam));
        acc += H[1] / (-lam + interp_odd(w, tb.invh, g.N, gam, -lam));
        dgam[n] = -acc / (2.0 * kPi);
    }
}

template <typename T>
__global__ void k_sigma_rhs_tri(Geo g, Tabs tb, TabsT tt, const double* __restrict__ w, const T* __restrict__ gam,
                                const T* __restrict__ G, double lam, T* __restrict__ dgam) {
    sigma_rhs_tri_block<T>(g, tb, tt, w, gam, G, lam, dgam, blockIdx.x);
}

// Shared-memory slot of component c of site r in a row: the 16 components of a site are
// stored XOR-rotated by the site index, so that lanes reading the same component of different
// sites (site-local products, lattice-sum entries) fall into different banks.
__host__ __device__ inline int tri_slot(int r, int c) { return r * 16 + (c ^ (r & 15)); }

// Site-local products of the s (CH = 0) or u (CH = 2) channel at one node, accumulated into
// o[16] (A, B: the site's two rows, rotated by sw = r & 15).
template <int CH, typename R>
__device__ __forceinline__ void tri_su_acc(const R* __restrict__ A, const R* __restrict__ B, int sw, R* o) {
    R a[16], b[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) { a[k] = A[k ^ sw]; b[k] = B[k ^ sw]; }
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
#pragma unroll
        for (int nu = 0; nu < 4; ++nu)
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const int cf = CH == 0 ? sr::tri::coef_s(mu, nu, x, y) : sr::tri::coef_u(mu, nu, x, y);
                    const R p = b[(x ^ mu) * 4 + (y ^ nu)];
                    o[mu * 4 + nu] = fmadd(cf > 0 ? a[x * 4 + y] : -a[x * 4 + y], p, o[mu * 4 + nu]);
                }
}

// t-channel on-site terms: A C (C the on-site row of the pair (i2, i2)) and D B (D of (i1, i1)).
template <typename R>
__device__ __forceinline__ void tri_onsite_acc(const R* __restrict__ A, const R* __restrict__ B, const R* __restrict__ C,
                                               const R* __restrict__ D, int sw, R* o) {
    R a[16], b[16], c[16], d[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) { a[k] = A[k ^ sw]; b[k] = B[k ^ sw]; c[k] = C[k]; d[k] = D[k]; }
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
#pragma unroll
        for (int nu = 0; nu < 4; ++nu)
#pragma unroll
            for (int l = 0; l < 4; ++l)
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int c2 = sr::tri::coef_o2(mu, nu, l, m);
                    const int c3 = sr::tri::coef_o3(mu, nu, l, m);
                    const R x2 = c[m * 4 + (m ^ l ^ nu)];
                    o[mu * 4 + nu] = fmadd(c2 > 0 ? a[mu * 4 + l] : -a[mu * 4 + l], x2, o[mu * 4 + nu]);
                    const R x3 = d[(mu ^ l ^ m) * 4 + l];
                    o[mu * 4 + nu] = fmadd(c3 > 0 ? x3 : -x3, b[m * 4 + nu], o[mu * 4 + nu]);
                }
}

template <typename R>
struct ShT {
    Desc<typename WeightOf<R>::type>* desc;   // kQTri * 4
    R* wq;                // kQTri * 4: node weights of rows 0 and 3 (dual numbers only; otherwise
                          // folded into the corner weights)
    int* mneg;            // kQTri * 4
    R* rows;              // kQTri * 2 * 16 Ns (site-major, component c of site r at tri_slot(r, c))
    R* onrow;             // kQTri * 2 * 16
    R* part;              // NG * Ns * 16: per node-group partial sums of the site-local products
    R* lat;               // lattice-sum integrals: per work item (FP32, n_items * 16) or per
                          // output (FP64, Ns * 16)
};

// Lattice-sum slots of k_gamma_rhs_tri<R>: FP32 work items, FP64 outputs.
__host__ __device__ inline int tri_lat_slots(int Ns, int n_items, size_t rsz) { return rsz == sizeof(float) ? n_items : Ns; }

// Dynamic shared memory of k_gamma_rhs_tri<R> (rsz = sizeof(R)).
__host__ __device__ inline size_t tri_smem_bytes(int Ns, int NG, int n_items, size_t rsz) {
    auto rnd = [](size_t b) { return (b + 15) & ~size_t(15); };
    const size_t dsz = rsz == sizeof(float) ? sizeof(Desc<float>) : sizeof(Desc<double>);
    return rnd(dsz * kQTri * 4) + (rsz > sizeof(double) ? rnd(rsz * kQTri * 4) : 0) + rnd(sizeof(int) * kQTri * 4) +
           rnd(rsz * kQTri * 2 * 16 * Ns) +
           rnd(rsz * kQTri * 2 * 16) + rnd(rsz * (size_t)NG * Ns * 16) + rnd(rsz * (size_t)tri_lat_slots(Ns, n_items, rsz) * 16);
}

// Lattice sum of one work item at the nodes of the current block: for every table entry of the
// item, the 4 x 4 spin matrices A (rows of (ref, j)) and B (rows of (j, i2)) under their signed
// component maps, out^{mu nu} += sum_l sign(mu, l, nu) A^{mu l} B^{l nu} (the factor 2 and the
// leading minus are applied at the end).  The signs of a signed permutation factorise,
// sign A^{mu l} = alpha(mu) beta(l) and sign B^{l nu} = gamma(l) delta(nu): the node sums run
// on unsigned loads with beta(l) gamma(l) on B, and alpha(mu) delta(nu) multiplies the entry's
// sum once (codes: row slots in bits 0..14; bit 15 of code mu = alpha(mu) < 0, of code 4 + nu =
// delta(nu) < 0, of code 8 + l = beta(l) gamma(l) < 0).
template <typename R>
__device__ __forceinline__ void tri_lattice_item(const R* __restrict__ rows, int row, int qn, const uint4* __restrict__ rec,
                                                 int e0, int e1, R* acc) {
    for (int e = e0; e < e1; ++e) {
        const uint4 w0 = rec[4 * e], w1 = rec[4 * e + 1], w2 = rec[4 * e + 2], w3 = rec[4 * e + 3];
        const unsigned wd[16] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w,
                                 w2.x, w2.y, w2.z, w2.w, w3.x, w3.y, w3.z, w3.w};
        int off[32];
        R sg[12];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const unsigned c = (k & 1) ? (wd[k >> 1] >> 16) : (wd[k >> 1] & 0xffffu);
            off[k] = (int)(c & 0x7fffu);
            if (k < 12) sg[k] = (c & 0x8000u) ? R(-1) : R(1);
        }
        R t[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) t[k] = R(0);
        for (int q = 0; q < qn; ++q) {
            const R* Ar = rows + (q * 2) * row;
            const R* Br = Ar + row;
            R a[16], b[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                a[k] = Ar[off[k]];
                b[k] = Br[off[16 + k]] * sg[8 + (k >> 2)];
            }
#pragma unroll
            for (int mu = 0; mu < 4; ++mu)
#pragma unroll
                for (int nu = 0; nu < 4; ++nu)
#pragma unroll
                    for (int l = 0; l < 4; ++l)
                        t[mu * 4 + nu] = fmadd(sr::tri::coef_t(mu, nu, l) > 0 ? a[mu * 4 + l] : -a[mu * 4 + l], b[l * 4 + nu],
                                               t[mu * 4 + nu]);
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu)
#pragma unroll
            for (int nu = 0; nu < 4; ++nu) acc[mu * 4 + nu] = fmadd(sg[mu] * sg[4 + nu], t[mu * 4 + nu], acc[mu * 4 + nu]);
    }
}

__host__ __device__ inline int tri_groups(int Ns, int threads) {
    const int ng = threads / Ns;
    return ng < 1 ? 1 : (ng > kQTri ? kQTri : ng);
}

// dGamma/dLambda of every stored entry of one frequency triple (one CTA per triple).  R is
// the type of the state read (the FP64 state, or its FP32 copy), of the lookup weights, the
// interpolated rows, the products and their node sums (double: FP64 flow; float: FP32-mixed
// flow, output in FP64; DualT: the tangent-linear flow, FP64 descriptors with the node weights
// applied to the rows).
template <typename R> using TriOut = typename std::conditional<std::is_same<R, float>::value, double, R>::type;

template <typename R>
__global__ void __launch_bounds__(kThreads) k_gamma_rhs_tri(Geo g, Tabs tb, TabsT tt, const double* __restrict__ w,
                                                            const R* __restrict__ G, const double* __restrict__ nx,
                                                            const TriOut<R>* __restrict__ nW, const int* __restrict__ ncount,
                                                            TriOut<R>* __restrict__ dG, int p0) {
    using D = typename WeightOf<R>::type;                 // descriptor weights
    constexpr bool kFold = std::is_same<D, R>::value;     // node weights folded into the corner weights
    constexpr bool kF32 = std::is_same<R, float>::value;
    extern __shared__ __align__(16) unsigned char smem[];
    const int NG = tri_groups(g.Ns, blockDim.x);
    ShT<R> sh;
    {
        size_t off = 0;
        auto take = [&](size_t bytes) { unsigned char* q = smem + off; off += (bytes + 15) & ~size_t(15); return q; };
        sh.desc = (Desc<D>*)take(sizeof(Desc<D>) * kQTri * 4);
        sh.wq = kFold ? nullptr : (R*)take(sizeof(R) * kQTri * 4);
        sh.mneg = (int*)take(sizeof(int) * kQTri * 4);
        sh.rows = (R*)take(sizeof(R) * kQTri * 2 * 16 * g.Ns);
        sh.onrow = (R*)take(sizeof(R) * kQTri * 2 * 16);
        sh.part = (R*)take(sizeof(R) * (size_t)NG * g.Ns * 16);
        sh.lat = (R*)take(sizeof(R) * (size_t)tri_lat_slots(g.Ns, tt.n_items, sizeof(R)) * 16);
    }
    const int tid = threadIdx.x;
    const int ti = blockIdx.x % g.N;
    const int p = p0 + (int)(blockIdx.x / g.N);   // stored pairs p0, p0 + 1, ...
    int si = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
    while ((si + 1) * (si + 2) / 2 <= p) ++si;
    while (si * (si + 1) / 2 > p) --si;
    const int ui = p - si * (si + 1) / 2;
    const double s = w[si], t = w[ti], u = w[ui];
    const double w1p = (s + t + u) / 2, w2p = (s - t - u) / 2, w1 = (s - t + u) / 2, w2 = (s + t - u) / 2;
    const int row = g.Ns * 16;
    const int nwork = g.Ns * NG;

    for (int o = tid; o < NG * row; o += blockDim.x) sh.part[o] = R(0);
    for (int o = tid; o < tri_lat_slots(g.Ns, tt.n_items, sizeof(R)) * 16; o += blockDim.x) sh.lat[o] = R(0);

    // row entries e = tid + k blockDim.x (e = c Ns + r: component c of site r) of this thread,
    // when they fit in registers: the shared-memory slot, the plain read (offset c Ns + r in
    // the entry block of a corner; bit 30: density weights, bit 29: imaginary-class function)
    // and the read through the site exchange (offset of the mapped component and site; bit
    // 30: density weights, bit 28: sign of the map)
    constexpr int kRE = 8;
    const bool rows_reg = row <= kRE * (int)blockDim.x;
    int e_slot[kRE], e_pl[kRE], e_sw[kRE];
#pragma unroll
    for (int k = 0; k < kRE; ++k) {
        const int e = tid + k * (int)blockDim.x;
        e_slot[k] = e_pl[k] = e_sw[k] = 0;
        if (rows_reg && e < row) {
            const int c = e / g.Ns, r = e - c * g.Ns;
            e_slot[k] = tri_slot(r, c);
            e_pl[k] = (c * g.Ns + r) | (((c & 3) == 0) << 30) | ((int)tri_mixed(c) << 29);
            const int m = tt.swap_map[c * g.Ns + r], cs = m & 15;
            e_sw[k] = (cs * g.Ns + tb.swap_r[r]) | (((cs & 3) == 0) << 30) | (((m & 16) != 0) << 28);
        }
    }

    for (int ch = 0; ch < 3; ++ch) {
        const int vi = ch == 0 ? si : (ch == 1 ? ti : ui);
        const int cidx = ch * g.N + vi;
        const int nq = ncount[cidx];
        const double* X = nx + (size_t)cidx * g.nmax;
        const TriOut<R>* Wp = nW + (size_t)cidx * g.nmax;
        const int nrow = ch == 1 ? 4 : 2;
        for (int q0 = 0; q0 < nq; q0 += kQTri) {
            const int qn = min(kQTri, nq - q0);
            __syncthreads();
            // descriptors of every row at every node of this block; the node weight goes into
            // the corner weights of the first row (and of the second on-site row)
            for (int idx = tid; idx < qn * nrow; idx += blockDim.x) {
                const int q = idx / nrow, rw = idx % nrow;
                const double x = X[q0 + q];
                double a, b, c;
                node_args(ch, rw, x, s, t, u, w1p, w2p, w1, w2, a, b, c);
                const int exs = ch == 0 ? 0 : (ch == 2 ? 2 : (rw < 2 ? 1 : 2));
                Desc<D>& d = sh.desc[q * 4 + rw];
                sh.mneg[q * 4 + rw] = (b < 0.0) != (c < 0.0);
                if constexpr (kFold) {
                    // the node weight goes into the corner weights of rows 0 and 3
                    make_desc<D, true>(a, b, c, exs, vi, tb, g, d, (rw == 0 || rw == 3) ? (D)Wp[q0 + q] : D(1));
                } else {
                    make_desc(a, b, c, exs, vi, tb, g, d);
                    if (rw == 0 || rw == 3) sh.wq[q * 4 + rw] = Wp[q0 + q];
                }
            }
            __syncthreads();
            // rows, with the sites fastest so that a warp reads consecutive sites of one stored
            // component (coalesced corner loads)
            if (rows_reg) {
                // every thread owns the same row entries at every node: descriptor in registers
                // per (node, row), entry maps resolved once per CTA
                for (int qr = 0; qr < qn * 2; ++qr) {
                    const int dq = (qr >> 1) * 4 + (qr & 1);
                    const Desc<D>& d = sh.desc[dq];
                    const int n = d.n, sw = d.swap, mn = sh.mneg[dq];
                    int o[4];
                    D wd[4], ws[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) { o[j] = d.off[j]; wd[j] = d.wd[j]; ws[j] = d.ws[j]; }
                    R* dst = sh.rows + qr * row;
#pragma unroll
                    for (int k = 0; k < kRE; ++k)
                        if (tid + k * (int)blockDim.x < row) {
                            const int pe = sw ? e_sw[k] : e_pl[k];
                            const R* src = G + (pe & 0x0fffffff);
                            const bool dens = (pe >> 30) & 1;
                            R acc = R(0);
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if (j < n) acc = fmadd((R)src[o[j]], dens ? wd[j] : ws[j], acc);
                            if constexpr (!kFold)
                                if ((qr & 1) == 0) acc = acc * sh.wq[(qr >> 1) * 4];
                            const bool neg = (sw && ((e_sw[k] >> 28) & 1)) != (mn && ((e_pl[k] >> 29) & 1));
                            dst[e_slot[k]] = neg ? -acc : acc;
                        }
                }
            } else {
                // a thread's item (node q, row rw, component c, site r) advances by blockDim.x
                // without divisions
                int qr = tid / row;                         // q * 2 + rw
                int c = (tid - qr * row) / g.Ns;
                int r = tid - qr * row - c * g.Ns;
                const int dc = (int)blockDim.x / g.Ns, dr = (int)blockDim.x - dc * g.Ns;
                for (int idx = tid; idx < qn * 2 * row; idx += blockDim.x) {
                    const int dq = (qr >> 1) * 4 + (qr & 1);
                    R v = tri_value<D>(G, sh.desc[dq], sh.mneg[dq] != 0, tb, tt, g, r, c);
                    if constexpr (!kFold)
                        if ((qr & 1) == 0) v = v * sh.wq[(qr >> 1) * 4];
                    sh.rows[qr * row + tri_slot(r, c)] = v;
                    r += dr;
                    c += dc;
                    if (r >= g.Ns) { r -= g.Ns; ++c; }
                    while (c >= 16) { c -= 16; ++qr; }
                }
            }
            if (ch == 1)
                for (int j = tid; j < qn * 2 * 16; j += blockDim.x) {
                    const int q = j / 32, rr = (j / 16) % 2, c = j % 16;
                    R v = tri_value<D>(G, sh.desc[q * 4 + 2 + rr], sh.mneg[q * 4 + 2 + rr] != 0, tb, tt, g, 0, c);
                    if constexpr (!kFold)
                        if (rr == 1) v = v * sh.wq[q * 4 + 3];
                    sh.onrow[(q * 2 + rr) * 16 + c] = v;
                }
            __syncthreads();
            // site-local products: work item (site r, node group gq) owns part[gq][r]
            for (int wk = tid; wk < nwork; wk += blockDim.x) {
                const int r = wk % g.Ns, gq = wk / g.Ns;
                R o[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) o[k] = R(0);
                for (int q = gq; q < qn; q += NG) {
                    const R* A = sh.rows + (q * 2) * row + r * 16;
                    const R* B = A + row;
                    if (ch == 0) tri_su_acc<0, R>(A, B, r & 15, o);
                    else if (ch == 2) tri_su_acc<2, R>(A, B, r & 15, o);
                    else {
                        R Cp[16];
                        const R* C0 = sh.onrow + (q * 2) * 16;
#pragma unroll
                        for (int k = 0; k < 16; ++k) {
                            const int mk = tt.onsite_map[r * 16 + k];
                            Cp[k] = (mk & 16) ? -C0[mk & 15] : C0[mk & 15];
                        }
                        tri_onsite_acc<R>(A, B, Cp, sh.onrow + (q * 2 + 1) * 16, r & 15, o);
                    }
                }
                R* P = sh.part + (size_t)gq * row + r * 16;
#pragma unroll
                for (int k = 0; k < 16; ++k) P[k] += o[k];
            }
            // lattice sum.  FP32: work items (a site and a chunk of its table entries), one per
            // thread, 4 x 4 spin matrices per entry (half a shared-memory load per FMA); FP64
            // (bound by the FP64 pipe): every output (site, component) integrates its signed
            // products
            if (ch == 1 && !kF32)
                for (int o = tid; o < row; o += blockDim.x) {
                    // four products at a time: independent FMA chains over the nodes
                    R acc = R(0);
                    const int k0 = tt.lat_off[o], k1 = tt.lat_off[o + 1];
                    int k = k0;
                    for (; k + 4 <= k1; k += 4) {
                        int ia[4], ib[4];
                        bool ng[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int2 en = tt.lat_ent[k + j];
                            ng[j] = en.y < 0;
                            ia[j] = en.x;
                            ib[j] = ng[j] ? ~en.y : en.y;
                        }
                        R a[4] = {R(0), R(0), R(0), R(0)};
                        for (int q = 0; q < qn; ++q) {
                            const R* Ar = sh.rows + (q * 2) * row;
                            const R* Br = Ar + row;
#pragma unroll
                            for (int j = 0; j < 4; ++j) a[j] = fmadd(Ar[ia[j]], Br[ib[j]], a[j]);
                        }
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc += ng[j] ? -a[j] : a[j];
                    }
                    for (; k < k1; ++k) {
                        const int2 en = tt.lat_ent[k];
                        const int ib = en.y < 0 ? ~en.y : en.y;
                        R a = R(0);
                        for (int q = 0; q < qn; ++q) a = fmadd(sh.rows[(q * 2) * row + en.x], sh.rows[(q * 2 + 1) * row + ib], a);
                        acc += en.y < 0 ? -a : a;
                    }
                    sh.lat[o] += acc;
                }
            if constexpr (kF32) {
                if (ch == 1)
                    for (int it = tid; it < tt.n_items; it += blockDim.x) {
                        const int4 item = tt.lat_items[it];
                        R acc[16];
#pragma unroll
                        for (int k = 0; k < 16; ++k) acc[k] = R(0);
                        tri_lattice_item<R>(sh.rows, row, qn, tt.lat_rec, item.y, item.z, acc);
                        R* L = sh.lat + (size_t)it * 16;
#pragma unroll
                        for (int k = 0; k < 16; ++k) L[k] += acc[k];
                    }
            }
        }
    }
    __syncthreads();
    for (int o = tid; o < row; o += blockDim.x) {
        R a = R(0);
        for (int k = 0; k < NG; ++k) a += sh.part[(size_t)k * row + o];
        const int r = o >> 4, c = o & 15;
        R l = R(0);
        if constexpr (!kF32) l = sh.lat[o];
        else
            for (int it = tt.lat_item_off[r]; it < tt.lat_item_off[r + 1]; ++it) l += sh.lat[(size_t)it * 16 + c];
        dG[((size_t)(p * g.N + ti) * 16 + c) * g.Ns + r] = TriOut<R>(a) - 2.0 * TriOut<R>(l);
    }
}

// FP32 copy of the TRI state (same layout) for the FP32-mixed vertex kernel.
__global__ void k_shadow_tri(long n, const double* __restrict__ G, float* __restrict__ Gf) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) Gf[i] = (float)G[i];
}

// Correlations chi^{mu nu}_{b j}, all 16 components (Eq. frg:correlation), one block per
// (b, j): bubble delta_{mu nu} (local) and the product-trapezoid vertex term.  T: double, or
// the dual numbers of a tangent flow.
template <typename T>
__global__ void k_chi_tri(Geo g, Tabs tb, TabsT tt, const double* __restrict__ w, const T* __restrict__ gam,
                          const T* __restrict__ G, double lam, const int* __restrict__ cr,
                          const int* __restrict__ cm, const int* __restrict__ onsite, int ntot, T* __restrict__ chi) {
    __shared__ double y[kMaxFreq + 1];
    __shared__ __align__(16) unsigned char wn_raw[sizeof(T) * (kMaxFreq + 1)];
    __shared__ double red[16 * 32 * (sizeof(T) / sizeof(double))];
    __shared__ int Ksh;
    T* Wn = reinterpret_cast<T*>(wn_raw);
    const int pidx = blockIdx.x;      // b * ntot + j
    const int b = pidx / ntot;
    const int on = onsite[pidx];
    const int r = cr[pidx];
    const int r0 = cr[b * ntot];      // the first site of each list is (0, b) itself
    const int* m = cm + (size_t)pidx * 16;
    const int* m0 = cm + (size_t)b * ntot * 16;
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
    T acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = T(0.0);
    for (int idx = threadIdx.x; idx < M * M; idx += blockDim.x) {
        const int pi = idx / M, qi = idx % M;
        const double xp = pi < K ? y[pi] : -y[pi - K];
        const double xq = qi < K ? y[qi] : -y[qi - K];
        const T wpq = Wn[pi % K] * Wn[qi % K];
        Desc<double> d;
        make_desc(xp + xq, 0.0, xp - xq, 1, 0, tb, g, d);
        const bool mn = (xp - xq) < 0.0;
        T v[16], e[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int mc = m[c];
            const T x = tri_value(G, d, mn, tb, tt, g, r, mc & 15);
            v[c] = (mc & 16) ? -x : x;
        }
        if (on) {
            make_desc(xp + xq, xq - xp, 0.0, 2, 0, tb, g, d);
            const bool me = (xq - xp) < 0.0;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int mc = m0[c];
                const T x = tri_value(G, d, me, tb, tt, g, r0, mc & 15);
                e[c] = (mc & 16) ? -x : x;
            }
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu)
#pragma unroll
            for (int nu = 0; nu < 4; ++nu) {
                T F = 4.0 * v[mu * 4 + nu];
                if (on) {
                    T x = T(0.0);
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        const T ev = e[(mu ^ nu ^ l) * 4 + l];
                        x += sr::tri::coef_x(mu, nu, l) > 0 ? T(2.0 * ev) : T(-2.0 * ev);
                    }
                    F -= x;
                }
                acc[mu * 4 + nu] += wpq * F;
            }
    }
    block_sum<T, 16>(acc, red);
    if (threadIdx.x == 0) {
        T bub = T(0.0);
        for (int k = 0; k < K; ++k) bub += Wn[k];
        bub = bub / (2.0 * kPi);
        for (int c = 0; c < 16; ++c)
            chi[(size_t)pidx * 16 + c] = ((on && (c >> 2) == (c & 3)) ? bub : T(0.0)) - acc[c] / (16.0 * kPi * kPi);
    }
}

// chi(k) = (1/N_b) sum_{b, j} cos(k (r_b - r_j)) (chi^xx + chi^yy + chi^zz)_{b j}.
template <typename T>
__global__ void k_chi_k_tri(int nk, const double* __restrict__ kp, const T* __restrict__ chi,
                            const double* __restrict__ dr, int npairs, int nb, T* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nk) return;
    const double kx = kp[3 * i], ky = kp[3 * i + 1], kz = kp[3 * i + 2];
    T acc = T(0.0);
    for (int p = 0; p < npairs; ++p) {
        const T sp = chi[(size_t)p * 16 + 5] + chi[(size_t)p * 16 + 10] + chi[(size_t)p * 16 + 15];
        acc += cos(kx * dr[3 * p] + ky * dr[3 * p + 1] + kz * dr[3 * p + 2]) * sp;
    }
    out[i] = acc / (double)nb;
}

}  // namespace
