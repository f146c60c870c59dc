// FP32-mixed SU(2) vertex flow (internal header, included by flow.cu after the shared device
// helpers).
//
// The same equations as k_gamma_rhs (Eq. frg:flowexplicit:2particle, projected on the SU(2)
// basis: density d = Gamma^00, spin s = Gamma^zz), with FP32 rows, products and accumulation,
// organised for few instructions and few barriers per stored triple:
//   * per channel and block of integration nodes, one descriptor per (node, row) -- the
//     symmetry folding of Eq. (frg:parametrizationBasis2p) and the four trilinear corners of
//     Sec. 4.2 (one argument of every row is a mesh frequency) -- is built once in shared
//     memory, branch-free: the argument is clamped to the mesh (constant extrapolation) and
//     always bracketed by two mesh points, one of which may carry weight zero;
//   * the nodes of the block are split into runs of consecutive nodes ("streams"); per stream a
//     pair of threads (row A, row B) per group of four sites interpolates both components of
//     its row from the FP32 shadow (16-byte loads of the four corner rows);
//   * s and u channels: the two threads of a site group exchange half of their rows by
//     shuffles and each forms the site-local products of two sites in registers;
//   * t channel: the on-site terms are formed in registers by the row threads; the rows go to
//     shared memory for the lattice sum, the dense per-triple contraction
//     C_c[rA][rB] = sum over nodes of A_c[rA] B_c[rB] in 4 x 4 register tiles, gathered
//     through the lattice-sum table at the end;
//   * every thread keeps its partial sums of all three channels in registers; they are combined
//     once per triple, in a fixed order.
#pragma once

namespace su2f {

constexpr int kThreadsS = 128;   // largest CTA (threads per triple) of k_gamma_rhs_su2f
constexpr int kMinCtas = 6;      // resident CTAs of kThreadsS threads the register budget is sized for

// CTA size for a lattice: 64 threads when a row has at most 32 padded sites (more, smaller CTAs
// per SM: cheaper barriers, measured faster), else 128 (enough row threads per node block).
__host__ __device__ inline int threads_for(int nsp) { return nsp <= 32 ? 64 : kThreadsS; }

// Whether the row threads keep the four corners of their row in registers from node to node
// (a corner shared by consecutive nodes is loaded once): it saves L1 traffic but costs about
// 45 registers, which pays off for wide rows (long streams at 128 threads), not for narrow ones
// (measured: pyrochlore range 6, 48 sites, 13.8 -> 12.8 ms; square range 7, 20 sites,
// 1.54 -> 1.70 ms).
__host__ __device__ inline bool cache_for(int nsp) { return nsp > 32; }
constexpr int kMinCtasCached = 4;   // resident CTAs of kThreadsS threads for the cached variant

// Descriptor of one vertex row: the four corners (two mesh points along each interpolated axis)
// with their element offsets in the shadow [Gf | Gs] and weights.
struct __align__(16) DescS {
    int off[4];     // element offset of the corner row in the shadow [Gf | Gs]
    float wd[4];    // weight of the density component (sign of the s <-> u relation folded in)
    float ws[4];    // weight of the spin component
};

// Bracketing mesh points k, k + 1 of x on the FP32 mesh in shared memory and the linear weights
// of Sec. 4.2: the argument is clamped to [w_0, w_N-1] first (constant extrapolation), so there
// are always two corners, one of weight zero outside the mesh or at a mesh point.
__device__ __forceinline__ void axis2(const float* w, const float* invh, const Geo& g, float x, int& k, float& wlo,
                                      float& whi) {
    const int N = g.N;
    const float xc = fminf(fmaxf(x, w[0]), w[N - 1]);
    k = interval_guess(g, xc);
    while (k > 0 && xc < w[k]) --k;
    while (k < N - 2 && xc >= w[k + 1]) ++k;
    wlo = (w[k + 1] - xc) * invh[k];
    whi = (xc - w[k]) * invh[k];
}

// Descriptor of Gamma(s, t, u) with one exact argument (ex_slot 0 s, 1 t, 2 u: the mesh
// frequency w[ex_idx]): the symmetry relations bring the arguments to s, t, u >= 0, s >= u
// (s -> -s and u -> -u exchange the sites: the row is read from the exchanged shadow Gs); the
// two other axes give the four corners.  The exact axis after the fold is selected
// arithmetically, so lanes of a warp take one path.  wn multiplies every weight (the node
// weight of weighted rows).  SLOTS: corners in parity-slot order (for the register cache).
template <bool SLOTS = false>
__device__ __forceinline__ void make_desc_s(float s, float t, float u, int ex_slot, int ex_idx, int swap_off,
                                            const float* w, const float* invh, const Geo& g, int rowp, float wn,
                                            DescS* dst) {
    const bool swap = (s < 0.0f) != (u < 0.0f);
    t = fabsf(t);
    s = fabsf(s);
    u = fabsf(u);
    const bool flip = s < u;
    const float sh = flip ? u : s, uh = flip ? s : u;
    const int ea = (flip && ex_slot != 1) ? 2 - ex_slot : ex_slot;   // exact axis after the fold
    const int so = swap ? swap_off : 0;
    // free axes: (t, u) for ea = 0, (s, u) for ea = 1, (s, t) for ea = 2
    const float x0 = ea == 0 ? t : sh, x1 = ea == 2 ? t : uh;
    int k0, k1;
    float v0[2], v1[2];
    axis2(w, invh, g, x0, k0, v0[0], v0[1]);
    axis2(w, invh, g, x1, k1, v1[0], v1[1]);
    v0[0] *= wn;
    v0[1] *= wn;
    int off[4];
    float wd[4], ws[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int b0 = k & 1, b1 = k >> 1;
        const int i0 = k0 + b0, i1 = k1 + b1;
        const int js = ea == 0 ? ex_idx : i0;
        const int jt = ea == 1 ? ex_idx : (ea == 0 ? i0 : i1);
        const int ju = ea == 2 ? ex_idx : i1;
        const float wt = v0[b0] * v1[b1];
        const bool below = js < ju;            // corner read through the s <-> u relation
        const int hi = below ? ju : js, lo = below ? js : ju;
        off[k] = ((hi * (hi + 1) / 2 + lo) * g.N + jt) * rowp + so;
        wd[k] = (flip != below) ? -wt : wt;
        ws[k] = wt;
    }
    if (SLOTS) {
        // corner (b0, b1) has mesh-index parities (k0 ^ b0, k1 ^ b1) & 1: put it in slot
        // k ^ x, x = parities of corner (0, 0), so that a corner shared by consecutive nodes
        // keeps its slot (two layers of selects, static register indices)
        const bool q0 = k0 & 1, q1 = k1 & 1;
        int o1[4];
        float d1[4], s1[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            o1[j] = q0 ? off[j ^ 1] : off[j];
            d1[j] = q0 ? wd[j ^ 1] : wd[j];
            s1[j] = q0 ? ws[j ^ 1] : ws[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            off[j] = q1 ? o1[j ^ 2] : o1[j];
            wd[j] = q1 ? d1[j ^ 2] : d1[j];
            ws[j] = q1 ? s1[j ^ 2] : s1[j];
        }
    }
    *reinterpret_cast<int4*>(dst->off) = make_int4(off[0], off[1], off[2], off[3]);
    *reinterpret_cast<float4*>(dst->wd) = make_float4(wd[0], wd[1], wd[2], wd[3]);
    *reinterpret_cast<float4*>(dst->ws) = make_float4(ws[0], ws[1], ws[2], ws[3]);
}

// Value of the on-site row (both components) at (s, t, u) with one exact argument: four
// corners read from the shadow directly (the on-site pair is its own exchange).
__device__ __forceinline__ void onsite_values(float s, float t, float u, int ex_slot, int ex_idx, const float* w,
                                              const float* invh, const Geo& g, int rowp, const float* __restrict__ Gf,
                                              float wn, float& v0, float& v1) {
    DescS d;
    make_desc_s(s, t, u, ex_slot, ex_idx, 0, w, invh, g, rowp, wn, &d);
    float a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] = __ldg(Gf + d.off[k]);
        b[k] = __ldg(Gf + d.off[k] + g.nsp);
    }
    v0 = fmaf(d.wd[3], a[3], fmaf(d.wd[2], a[2], fmaf(d.wd[1], a[1], d.wd[0] * a[0])));
    v1 = fmaf(d.ws[3], b[3], fmaf(d.ws[2], b[2], fmaf(d.ws[1], b[1], d.ws[0] * b[0])));
}

__device__ __forceinline__ float4 wsum4(const float4 (&c)[4], const float4 w) {
    float4 r;
    r.x = fmaf(w.w, c[3].x, fmaf(w.z, c[2].x, fmaf(w.y, c[1].x, w.x * c[0].x)));
    r.y = fmaf(w.w, c[3].y, fmaf(w.z, c[2].y, fmaf(w.y, c[1].y, w.x * c[0].y)));
    r.z = fmaf(w.w, c[3].z, fmaf(w.z, c[2].z, fmaf(w.y, c[1].z, w.x * c[0].z)));
    r.w = fmaf(w.w, c[3].w, fmaf(w.z, c[2].w, fmaf(w.y, c[1].w, w.x * c[0].w)));
    return r;
}

// Shared-memory layout of one triple (sizes in bytes, 16-byte aligned blocks).
struct Layout {
    size_t mesh, desc, fac, rows, acc, cacc, total;
};

__host__ __device__ inline int streams(int nsp, int threads) { return threads / (nsp / 2); }

__host__ __device__ inline Layout layout(int N, int Ns, int nsp, int qb, int threads) {
    auto r16 = [](size_t b) { return (b + 15) & ~size_t(15); };
    Layout L;
    const size_t rowp = 2 * (size_t)nsp;
    const size_t ntile = 2 * (size_t)(nsp / 4) * (nsp / 4);
    const size_t scr_site = (size_t)streams(nsp, threads) * 2 * rowp;          // partials [stream][row][c][nsp]
    const size_t scr_tile = ntile <= (size_t)threads ? (threads / ntile) * ntile * 16 : 0;
    L.mesh = r16(sizeof(float) * 2 * N);
    L.desc = r16(sizeof(DescS) * qb * 2);
    L.fac = r16(sizeof(float) * qb * 4);
    const size_t rows_a = (size_t)qb * 2 * rowp, rows_b = scr_site > scr_tile ? scr_site : scr_tile;
    const size_t rows = sizeof(float) * (rows_a > rows_b ? rows_a : rows_b);
    L.rows = r16(rows);
    L.acc = r16(sizeof(float) * Ns * 2);
    L.cacc = r16(sizeof(float) * 2 * nsp * nsp);
    L.total = L.mesh + L.desc + L.fac + L.rows + L.acc + L.cacc;
    return L;
}

// One stored frequency triple (pair p, transfer index ti): all irreducible sites, both
// components, written to dG (FP64).  Gf: FP32 shadow (padded layout); the exchanged shadow
// starts swap_off floats later (swap_off = 0 when the site exchange is trivial).  qb:
// integration nodes per shared-memory block.  Needs blockDim.x >= nsp / 2 (one stream).
template <bool CACHE>
__device__ void triple(const Geo& g, const Tabs& tb, const float* __restrict__ Gf, const int swap_off,
                       const float* __restrict__ nx, const float* __restrict__ nW, const int* __restrict__ ncount,
                       double* __restrict__ dG, const int p, const int ti, unsigned char* smem, const int qb) {
    constexpr int NC = 2;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int nsp = g.nsp, nsp4 = nsp >> 2, rowp = NC * nsp;
    const Layout Ly = layout(g.N, g.Ns, nsp, qb, nth);
    float* wm = reinterpret_cast<float*>(smem);
    float* ih = wm + g.N;
    DescS* desc = reinterpret_cast<DescS*>(smem + Ly.mesh);
    float* fac = reinterpret_cast<float*>(smem + Ly.mesh + Ly.desc);
    float* rows = reinterpret_cast<float*>(smem + Ly.mesh + Ly.desc + Ly.fac);
    float* acc = reinterpret_cast<float*>(smem + Ly.mesh + Ly.desc + Ly.fac + Ly.rows);
    float* cacc = reinterpret_cast<float*>(smem + Ly.mesh + Ly.desc + Ly.fac + Ly.rows + Ly.acc);

    int si = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);   // guess, corrected below
    while ((si + 1) * (si + 2) / 2 <= p) ++si;
    while (si * (si + 1) / 2 > p) --si;
    const int ui = p - si * (si + 1) / 2;
    __syncthreads();   // shared memory of a previous triple (persistent callers) is consumed
    for (int i = tid; i < g.N; i += nth) {
        wm[i] = tb.wf[i];
        ih[i] = i + 1 < g.N ? tb.invhf[i] : 0.0f;
    }
    for (int o = tid; o < g.Ns * NC; o += nth) acc[o] = 0.0f;
    for (int o = tid; o < NC * nsp * nsp; o += nth) cacc[o] = 0.0f;
    __syncthreads();
    const float s = wm[si], t = wm[ti], u = wm[ui];
    const float w1p = (s + t + u) * 0.5f, w2p = (s - t - u) * 0.5f, w1 = (s - t + u) * 0.5f, w2 = (s + t - u) * 0.5f;

    // streams: unit (site group sg, row r), U = 2 nsp4 units per stream
    const int U = 2 * nsp4, S = nth / U;
    const int stream = tid / U, unit = tid % U;
    const bool in_stream = stream < S;
    const int sg = unit >> 1, r = unit & 1;
    const float* pb0 = Gf + 4 * sg;          // component 0 (density) of the site group
    const float* pb1 = Gf + nsp + 4 * sg;    // component 1 (spin)
    // tiles of the dense contraction: (component, 4 sites of A, 4 sites of B)
    const int ntile = NC * nsp4 * nsp4;
    const bool tile_reg = ntile <= nth;
    const int TG = tile_reg ? nth / ntile : 1;
    const int my_tile = tid % ntile, my_tg = tid / ntile;
    const bool tile_on = tile_reg && my_tg < TG;

    // partial outputs of this thread's sites over all channels: s and u channels (sites
    // 4 sg + 2 r + i, i < 2) and t channel (sites 4 sg + i, i < 4), both components
    float psu[NC][2], pt[NC][4];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        psu[c][0] = psu[c][1] = 0.0f;
        pt[c][0] = pt[c][1] = pt[c][2] = pt[c][3] = 0.0f;
    }
    for (int ch = 0; ch < 3; ++ch) {
        const int vi = ch == 0 ? si : (ch == 1 ? ti : ui);
        const int cidx = ch * g.N + vi;
        const int nq = ncount[cidx];
        const float* X = nx + (size_t)cidx * g.nmax;
        const float* Wp = nW + (size_t)cidx * g.nmax;
        const int nrow = ch == 1 ? 4 : 2;
        float a4[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) a4[i][j] = 0.0f;
        for (int q0 = 0; q0 < nq; q0 += qb) {
            const int qn = min(qb, nq - q0);
            __syncthreads();
            // phase 1: descriptors (rows A, B) and on-site factors (t channel rows C, D)
            for (int idx = tid; idx < qn * nrow; idx += nth) {
                const int rw = idx / qn, q = idx - rw * qn;   // row-major: a warp's lanes mostly share the row
                const float x = X[q0 + q];
                float a, b, c;
                node_args<float>(ch, rw, x, s, t, u, w1p, w2p, w1, w2, a, b, c);
                const int exs = ch == 0 ? 0 : (ch == 2 ? 2 : (rw < 2 ? 1 : 2));
                // the node weight rides on row A (all channels) and on the on-site row D
                const float wn = (rw == 0 || rw == 3) ? Wp[q0 + q] : 1.0f;
                if (rw < 2) {
                    make_desc_s<CACHE>(a, b, c, exs, vi, swap_off, wm, ih, g, rowp, wn, &desc[q * 2 + rw]);
                } else {
                    float v0, v1;
                    onsite_values(a, b, c, exs, vi, wm, ih, g, rowp, Gf, wn, v0, v1);
                    // on-site factors sum_k s(k, c) C_k: density d + 3 s, spin d - s
                    fac[q * 4 + (rw - 2) * 2 + 0] = v0 + 3.0f * v1;
                    fac[q * 4 + (rw - 2) * 2 + 1] = v0 - v1;
                }
            }
            __syncthreads();
            // phase 2: interpolation along the streams
            {
                const int L = (qn + S - 1) / S;
                const int qa = stream * L, qe = min(qa + L, qn);
                float4 c0[4], c1[4];   // corner rows of this thread's sites, both components
                int tag[4];            // CACHE: offset of the corner each slot holds
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    c0[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                    c1[k] = c0[k];
                    tag[k] = -1;
                }
                for (int j = 0; j < L; ++j) {
                    const int q = qa + j;
                    const bool act = in_stream && q < qe;
                    float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
                    if (act) {
                        const DescS& d = desc[q * 2 + r];
                        const int4 off = *reinterpret_cast<const int4*>(d.off);
                        const float4 wd = *reinterpret_cast<const float4*>(d.wd);
                        const float4 ws = *reinterpret_cast<const float4*>(d.ws);
                        const int o4[4] = {off.x, off.y, off.z, off.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (!CACHE || o4[k] != tag[k]) {
                                c0[k] = __ldg(reinterpret_cast<const float4*>(pb0 + o4[k]));
                                c1[k] = __ldg(reinterpret_cast<const float4*>(pb1 + o4[k]));
                                tag[k] = o4[k];
                            }
                        }
                        v0 = wsum4(c0, wd);
                        v1 = wsum4(c1, ws);
                    }
                    if (ch != 1) {
                        // exchange half of the rows: this thread keeps sites 2r, 2r + 1 of its
                        // group and receives the partner row there (the products are symmetric
                        // under A <-> B)
                        const float s0 = r ? v0.x : v0.z, s1 = r ? v0.y : v0.w;
                        const float s2 = r ? v1.x : v1.z, s3 = r ? v1.y : v1.w;
                        const float o0 = __shfl_xor_sync(0xffffffffu, s0, 1);
                        const float o1 = __shfl_xor_sync(0xffffffffu, s1, 1);
                        const float o2 = __shfl_xor_sync(0xffffffffu, s2, 1);
                        const float o3 = __shfl_xor_sync(0xffffffffu, s3, 1);
                        const float d0 = r ? v0.z : v0.x, d1 = r ? v0.w : v0.y;   // own density, sites 2r, 2r + 1
                        const float e0 = r ? v1.z : v1.x, e1 = r ? v1.w : v1.y;   // own spin
                        // s channel: (dd + 3 ss, ds + sd - 2 ss); u channel: (dd + 3 ss, ds + sd + 2 ss)
                        const float k2 = ch == 0 ? -2.0f : 2.0f;
                        const float q0s = e0 * o2, q1s = e1 * o3;
                        psu[0][0] = fmaf(d0, o0, fmaf(3.0f, q0s, psu[0][0]));
                        psu[0][1] = fmaf(d1, o1, fmaf(3.0f, q1s, psu[0][1]));
                        psu[1][0] = fmaf(d0, o2, fmaf(e0, o0, fmaf(k2, q0s, psu[1][0])));
                        psu[1][1] = fmaf(d1, o3, fmaf(e1, o1, fmaf(k2, q1s, psu[1][1])));
                    } else if (act) {
                        // on-site terms: A_c F_c(C) (row A) and F_c(D) B_c (row B)
                        const float f0 = fac[q * 4 + 2 * r], f1 = fac[q * 4 + 2 * r + 1];
                        pt[0][0] = fmaf(v0.x, f0, pt[0][0]);
                        pt[0][1] = fmaf(v0.y, f0, pt[0][1]);
                        pt[0][2] = fmaf(v0.z, f0, pt[0][2]);
                        pt[0][3] = fmaf(v0.w, f0, pt[0][3]);
                        pt[1][0] = fmaf(v1.x, f1, pt[1][0]);
                        pt[1][1] = fmaf(v1.y, f1, pt[1][1]);
                        pt[1][2] = fmaf(v1.z, f1, pt[1][2]);
                        pt[1][3] = fmaf(v1.w, f1, pt[1][3]);
                        float* dst = rows + (size_t)(q * 2 + r) * rowp + 4 * sg;
                        *reinterpret_cast<float4*>(dst) = v0;
                        *reinterpret_cast<float4*>(dst + nsp) = v1;
                    }
                }
            }
            if (ch == 1) {
                __syncthreads();
                // phase 3: lattice sum, dense contraction over the block's nodes
                if (tile_on) {
                    const int c = my_tile / (nsp4 * nsp4), ra = (my_tile / nsp4) % nsp4, rb = my_tile % nsp4;
                    for (int q = my_tg; q < qn; q += TG) {
                        const float4 av = *reinterpret_cast<const float4*>(rows + (q * 2) * rowp + c * nsp + 4 * ra);
                        const float4 bv = *reinterpret_cast<const float4*>(rows + (q * 2 + 1) * rowp + c * nsp + 4 * rb);
                        const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) a4[i][j] = fmaf(ar[i], br[j], a4[i][j]);
                    }
                } else if (!tile_reg) {
                    for (int tl = tid; tl < ntile; tl += nth) {
                        const int c = tl / (nsp4 * nsp4), ra = (tl / nsp4) % nsp4, rb = tl % nsp4;
                        float t4[4][4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) t4[i][j] = 0.0f;
                        for (int q = 0; q < qn; ++q) {
                            const float4 av = *reinterpret_cast<const float4*>(rows + (q * 2) * rowp + c * nsp + 4 * ra);
                            const float4 bv = *reinterpret_cast<const float4*>(rows + (q * 2 + 1) * rowp + c * nsp + 4 * rb);
                            const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                            for (int i = 0; i < 4; ++i)
#pragma unroll
                                for (int j = 0; j < 4; ++j) t4[i][j] = fmaf(ar[i], br[j], t4[i][j]);
                        }
                        float* cp = cacc + c * nsp * nsp + (4 * ra) * nsp + 4 * rb;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            float4 cv = *reinterpret_cast<float4*>(cp + i * nsp);
                            cv.x += t4[i][0]; cv.y += t4[i][1]; cv.z += t4[i][2]; cv.w += t4[i][3];
                            *reinterpret_cast<float4*>(cp + i * nsp) = cv;
                        }
                    }
                }
            }
        }
        if (ch == 1 && tile_reg) {
            // end of the t channel: combine the tile groups' contractions in a fixed order
            float* scr2 = rows;   // [tile group][16][tile]
            __syncthreads();
            if (tile_on) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) scr2[(my_tg * 16 + i * 4 + j) * ntile + my_tile] = a4[i][j];
            }
            __syncthreads();
            for (int e = tid; e < ntile * 16; e += nth) {
                const int tl = e % ntile, ij = e / ntile;
                float a = 0.0f;
                for (int k = 0; k < TG; ++k) a += scr2[(k * 16 + ij) * ntile + tl];
                const int c = tl / (nsp4 * nsp4), ra = (tl / nsp4) % nsp4, rb = tl % nsp4;
                cacc[c * nsp * nsp + (4 * ra + (ij >> 2)) * nsp + 4 * rb + (ij & 3)] += a;
            }
        }
    }
    // end of the triple: combine the threads' partials in a fixed order (scratch: the row buffer)
    __syncthreads();
    float* scr = rows;   // [stream][row][c][nsp]
    if (in_stream) {
        float* o = scr + (size_t)(stream * 2 + r) * rowp + 4 * sg;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            float4 v = make_float4(pt[c][0], pt[c][1], pt[c][2], pt[c][3]);
            // s / u partials belong to sites 2r, 2r + 1 of the group
            if (r) { v.z += psu[c][0]; v.w += psu[c][1]; }
            else { v.x += psu[c][0]; v.y += psu[c][1]; }
            *reinterpret_cast<float4*>(o + c * nsp) = v;
        }
    }
    __syncthreads();
    for (int o = tid; o < g.Ns * NC; o += nth) {
        const int rr = o / NC, c = o % NC;
        float a = 0.0f;
        for (int k = 0; k < S * 2; ++k) a += scr[(size_t)k * rowp + c * nsp + rr];
        acc[o] = a;
    }
    __syncthreads();
    for (int o = tid; o < g.Ns * NC; o += nth) {
        const int rr = o / NC, c = o % NC;
        float a = 0.0f;
        for (int k = tb.gath_off[o]; k < tb.gath_off[o + 1]; ++k) a += cacc[tb.dgath_idx[k]];
        dG[((size_t)(p * g.N + ti) * NC + c) * g.Ns + rr] = (double)acc[o] - 2.0 * (double)a;
    }
}

}  // namespace su2f

// FP32-mixed SU(2) vertex flow, one CTA per stored frequency triple (CACHE: corner rows kept in
// registers from node to node).
template <bool CACHE>
__global__ void __launch_bounds__(su2f::kThreadsS, CACHE ? su2f::kMinCtasCached : su2f::kMinCtas)
k_gamma_rhs_su2f(Geo g, Tabs tb, const float* __restrict__ Gf, int swap_off,
                                                             const float* __restrict__ nx, const float* __restrict__ nW,
                                                             const int* __restrict__ ncount, double* __restrict__ dG, int qb,
                                                             int p0) {
    extern __shared__ __align__(16) unsigned char smem[];
    su2f::triple<CACHE>(g, tb, Gf, swap_off, nx, nW, ncount, dG, p0 + (int)(blockIdx.x / g.N), blockIdx.x % g.N, smem, qb);
}
