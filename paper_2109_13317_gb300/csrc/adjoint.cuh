// Reverse-mode (adjoint) kernels of the FP64 flow right-hand side and of the correlation
// measurement.  Included by flow.cu after the forward kernels, whose helpers (propagators,
// node arguments, channel products, lookup descriptors) they share.
//
// For the state y = (gamma, Gamma) and the right-hand side f(Lambda, y) of Sec. 3 (Eqs.
// frg:flowexplicit:1particle and frg:flowexplicit:2particle, discretised as in Sec. 4.2), the
// kernels compute the vector-Jacobian product ybar = (df/dy)^T fbar.  f is evaluated in three
// stages -- dgamma (k_sigma_rhs), the integration nodes and weights W(gamma, dgamma)
// (k_channel_nodes), and dGamma = sum_nodes W * (bilinear vertex products) (k_gamma_rhs) --
// and the adjoint runs them backwards:
//   k_gamma_adj  Gammabar += (d dGamma / d Gamma)^T fbar_Gamma,  Wbar = d dGamma / d W . fbar_Gamma
//   k_nodes_adj  gammabar += (dW / d gamma)^T Wbar,  dgammabar += (dW / d dgamma)^T Wbar
//   k_sigma_adj  with dgammabar + fbar_gamma: Gammabar and gammabar through dgamma(gamma, Gamma)
// Every transposed lookup scatters into the state with atomic additions (the forward gathers
// read arbitrary entries), so sums are formed in a run-dependent order: results agree with an
// exact evaluation to rounding, not bit for bit between runs.
#pragma once

namespace {

// Inverted lattice-sum tables (host-built from the product list and its gather table).
struct AdjTabs {
    const int* pinv_off;   // nprod + 1: outputs using each product
    const int* pinv_out;   // output index r * nc + c
    const int* ainv_off;   // Ns * nc + 1: products whose row-A index is e
    const int* ainv_idx;
    const int* binv_off;   // Ns * nc + 1: products whose row-B index is e
    const int* binv_idx;
};

// Transpose of interp_odd: scatter vbar = d/d gamma(x) onto the mesh values.
__device__ __forceinline__ void interp_odd_adj(const double* __restrict__ w, const double* __restrict__ invh, int N,
                                               double* __restrict__ fbar, double x, double vbar) {
    if (x == 0.0 || vbar == 0.0) return;
    int lo;
    double wl, wh;
    bracket(w, invh, N, fabs(x), lo, wl, wh);
    const double sg = x < 0.0 ? -1.0 : 1.0;
    if (wl != 0.0) atomicAdd(&fbar[lo], sg * wl * vbar);
    if (wh != 0.0) atomicAdd(&fbar[lo + 1], sg * wh * vbar);
}

// Transpose of row_value: scatter vbar = d/d(row value (r, c)) onto the stored corners.
__device__ __forceinline__ void row_value_adj(double* __restrict__ Gbar, const Desc<double>& d, const Tabs& tb,
                                              const Geo& g, int r, int c, double vbar) {
    if (vbar == 0.0) return;
    int rs = r, cs = c;
    if (d.swap) { rs = tb.swap_r[r]; cs = perm_of(tb.swap_perm[r], c); }
    double* base = Gbar + cs * g.Ns + rs;
    const double* wgt = c == 0 ? d.wd : d.ws;
    for (int k = 0; k < d.n; ++k)
        if (wgt[k] != 0.0) atomicAdd(base + d.off[k], wgt[k] * vbar);
}

struct AdjSh {
    Desc<double>* desc;
    double* rows;    // raw interpolated rows (no node weight)
    double* rbar;    // their adjoints
    double* onrow;
    double* onbar;
    double* wq;
    double* wb;      // adjoint of the node weights of the current block
    double* ob;      // fbar of this triple, index r * nc + c
    double* pbar;    // adjoint of each lattice-sum product integral
};

__host__ __device__ inline size_t adj_smem_bytes(int Ns, int nc, int nprod) {
    auto rnd = [](size_t b) { return (b + 15) & ~size_t(15); };
    const size_t row = (size_t)Ns * nc;
    return rnd(sizeof(Desc<double>) * kQC * 4) + 2 * rnd(sizeof(double) * kQC * 2 * row) +
           2 * rnd(sizeof(double) * kQC * 2 * nc) + 2 * rnd(sizeof(double) * kQC) + rnd(sizeof(double) * row) +
           rnd(sizeof(double) * nprod);
}

// Vertex part: one CTA per stored (s, u, t) triple, the node loop of k_gamma_rhs with every
// product differentiated.  For a node with weight W and raw rows A, B:
//   s / u channel  out_r += W prod(A_r, B_r)          (prod bilinear: dprod/dA_c = prod(e_c, B))
//   t channel      out_r += W [A_r . of(C) + of(D) . B_r] - 2 W sum_products A_x B_y
// so Abar, Bbar, Cbar, Dbar carry W, and Wbar collects the bracket contracted with fbar.
template <int NC>
__global__ void __launch_bounds__(kThreads) k_gamma_adj(Geo g, Tabs tb, AdjTabs at, const double* __restrict__ w,
                                                        const double* __restrict__ G, const double* __restrict__ nx,
                                                        const double* __restrict__ nW, const int* __restrict__ ncount,
                                                        const double* __restrict__ fbar, double* __restrict__ Gbar,
                                                        double* __restrict__ Wbar) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int row = g.Ns * NC;
    AdjSh sh;
    {
        size_t off = 0;
        auto take = [&](size_t bytes) { unsigned char* q = smem + off; off += (bytes + 15) & ~size_t(15); return q; };
        sh.desc = (Desc<double>*)take(sizeof(Desc<double>) * kQC * 4);
        sh.rows = (double*)take(sizeof(double) * kQC * 2 * row);
        sh.rbar = (double*)take(sizeof(double) * kQC * 2 * row);
        sh.onrow = (double*)take(sizeof(double) * kQC * 2 * NC);
        sh.onbar = (double*)take(sizeof(double) * kQC * 2 * NC);
        sh.wq = (double*)take(sizeof(double) * kQC);
        sh.wb = (double*)take(sizeof(double) * kQC);
        sh.ob = (double*)take(sizeof(double) * row);
        sh.pbar = (double*)take(sizeof(double) * tb.nprod);
    }
    const int tid = threadIdx.x;
    const int ti = blockIdx.x % g.N;
    const int p = blockIdx.x / g.N;
    int si = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
    while ((si + 1) * (si + 2) / 2 <= p) ++si;
    while (si * (si + 1) / 2 > p) --si;
    const int ui = p - si * (si + 1) / 2;
    const double s = w[si], t = w[ti], u = w[ui];
    const double w1p = (s + t + u) / 2, w2p = (s - t - u) / 2, w1 = (s - t + u) / 2, w2 = (s + t - u) / 2;

    for (int e = tid; e < row; e += blockDim.x) {
        const int r = e / NC, c = e % NC;
        sh.ob[e] = fbar[((size_t)(p * g.N + ti) * NC + c) * g.Ns + r];
    }
    __syncthreads();
    // out_o = acc_o - 2 sum_{products of o} part  =>  partbar = -2 sum_{outputs using it} fbar_o
    for (int o = tid; o < tb.nprod; o += blockDim.x) {
        double a = 0.0;
        for (int k = at.pinv_off[o]; k < at.pinv_off[o + 1]; ++k) a += sh.ob[at.pinv_out[k]];
        sh.pbar[o] = -2.0 * a;
    }

    for (int ch = 0; ch < 3; ++ch) {
        const int vi = ch == 0 ? si : (ch == 1 ? ti : ui);
        const int cidx = ch * g.N + vi;
        const int nq = ncount[cidx];
        const double* X = nx + (size_t)cidx * g.nmax;
        const double* Wp = nW + (size_t)cidx * g.nmax;
        const int nrow = ch == 1 ? 4 : 2;
        for (int q0 = 0; q0 < nq; q0 += kQC) {
            const int qn = min(kQC, nq - q0);
            __syncthreads();
            for (int idx = tid; idx < qn * nrow; idx += blockDim.x) {
                const int q = idx / nrow, rw = idx % nrow;
                const double x = X[q0 + q];
                double a, b, c;
                node_args(ch, rw, x, s, t, u, w1p, w2p, w1, w2, a, b, c);
                const int exs = ch == 0 ? 0 : (ch == 2 ? 2 : (rw < 2 ? 1 : 2));
                make_desc(a, b, c, exs, vi, tb, g, sh.desc[q * 4 + rw]);
                if (rw == 0) { sh.wq[q] = Wp[q0 + q]; sh.wb[q] = 0.0; }
            }
            for (int j = tid; j < qn * 2 * NC; j += blockDim.x) sh.onbar[j] = 0.0;
            __syncthreads();
            for (int idx = tid; idx < qn * 2 * row; idx += blockDim.x) {
                const int q = idx / (2 * row), rem = idx % (2 * row), rw = rem / row, e = rem % row;
                sh.rows[idx] = row_value(G, sh.desc[q * 4 + rw], tb, g, e / NC, e % NC);
            }
            if (ch == 1)
                for (int j = tid; j < qn * 2 * NC; j += blockDim.x) {
                    const int qq = j / (2 * NC), rr = (j / NC) % 2, c = j % NC;
                    sh.onrow[j] = row_value(G, sh.desc[qq * 4 + 2 + rr], tb, g, 0, c);
                }
            __syncthreads();
            for (int item = tid; item < qn * g.Ns; item += blockDim.x) {
                const int q = item / g.Ns, r = item % g.Ns;
                const double* A = sh.rows + (q * 2) * row + r * NC;
                const double* B = sh.rows + (q * 2 + 1) * row + r * NC;
                const double* o = sh.ob + r * NC;
                const double W = sh.wq[q];
                double Ab[NC], Bb[NC], E[NC], out[NC];
                double wsum = 0.0;
                if (ch != 1) {
#pragma unroll
                    for (int k = 0; k < NC; ++k) {
#pragma unroll
                        for (int c = 0; c < NC; ++c) E[c] = c == k ? 1.0 : 0.0;
                        if (ch == 0) s_product<double, NC>(E, B, out); else u_product<double, NC>(E, B, out);
                        double a = 0.0;
#pragma unroll
                        for (int c = 0; c < NC; ++c) a += o[c] * out[c];
                        Ab[k] = a;
                        if (ch == 0) s_product<double, NC>(A, E, out); else u_product<double, NC>(A, E, out);
                        a = 0.0;
#pragma unroll
                        for (int c = 0; c < NC; ++c) a += o[c] * out[c];
                        Bb[k] = a;
                    }
                    if (ch == 0) s_product<double, NC>(A, B, out); else u_product<double, NC>(A, B, out);
#pragma unroll
                    for (int c = 0; c < NC; ++c) wsum += o[c] * out[c];
                } else {
                    const int pon = tb.onsite_perm[r];
                    const double* C0 = sh.onrow + (q * 2) * NC;
                    const double* D = sh.onrow + (q * 2 + 1) * NC;
                    double Cp[NC];
#pragma unroll
                    for (int k = 0; k < NC; ++k) Cp[k] = C0[perm_of(pon, k)];
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const double fc = onsite_factor<double, NC>(Cp, c), fd = onsite_factor<double, NC>(D, c);
                        Ab[c] = o[c] * fc;
                        Bb[c] = o[c] * fd;
                        wsum += o[c] * (A[c] * fc + fd * B[c]);
                    }
                    // on-site rows: of() is linear, d of(C, c) / d C_k = of(e_k, c)
#pragma unroll
                    for (int k = 0; k < NC; ++k) {
#pragma unroll
                        for (int c = 0; c < NC; ++c) E[c] = c == k ? 1.0 : 0.0;
                        double cb = 0.0, db = 0.0;
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            const double fe = onsite_factor<double, NC>(E, c);
                            cb += o[c] * A[c] * fe;
                            db += o[c] * B[c] * fe;
                        }
                        if (cb != 0.0) atomicAdd(&sh.onbar[(q * 2) * NC + perm_of(pon, k)], W * cb);
                        if (db != 0.0) atomicAdd(&sh.onbar[(q * 2 + 1) * NC + k], W * db);
                    }
                    // lattice sum
                    const double* Ar = sh.rows + (q * 2) * row;
                    const double* Br = sh.rows + (q * 2 + 1) * row;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const int e = r * NC + c;
                        double la = 0.0, lb = 0.0;
                        for (int k = at.ainv_off[e]; k < at.ainv_off[e + 1]; ++k) {
                            const int pr = at.ainv_idx[k];
                            la += sh.pbar[pr] * Br[tb.prod[pr].y];
                        }
                        for (int k = at.binv_off[e]; k < at.binv_off[e + 1]; ++k) {
                            const int pr = at.binv_idx[k];
                            lb += sh.pbar[pr] * Ar[tb.prod[pr].x];
                        }
                        Ab[c] += la;
                        Bb[c] += lb;
                        wsum += A[c] * la;
                    }
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    sh.rbar[(q * 2) * row + r * NC + c] = W * Ab[c];
                    sh.rbar[(q * 2 + 1) * row + r * NC + c] = W * Bb[c];
                }
                if (wsum != 0.0) atomicAdd(&sh.wb[q], wsum);
            }
            __syncthreads();
            for (int idx = tid; idx < qn * 2 * row; idx += blockDim.x) {
                const int q = idx / (2 * row), rem = idx % (2 * row), rw = rem / row, e = rem % row;
                row_value_adj(Gbar, sh.desc[q * 4 + rw], tb, g, e / NC, e % NC, sh.rbar[idx]);
            }
            if (ch == 1)
                for (int j = tid; j < qn * 2 * NC; j += blockDim.x) {
                    const int qq = j / (2 * NC), rr = (j / NC) % 2, c = j % NC;
                    row_value_adj(Gbar, sh.desc[qq * 4 + 2 + rr], tb, g, 0, c, sh.onbar[j]);
                }
            for (int q = tid; q < qn; q += blockDim.x)
                if (sh.wb[q] != 0.0) atomicAdd(&Wbar[(size_t)cidx * g.nmax + q0 + q], sh.wb[q]);
        }
    }
}

// Node weights: one block per (channel, transfer frequency).  Delta points carry
// W = gg(a, L) / 2pi with gg(a, b) = -1 / ((a + gamma_a)(b + gamma_b)); regular points carry
// W = tw * (gr(x, y) + gr(y, x)) / 2pi with gr(a, b) = -dgamma_b / ((a + gamma_a)(b + gamma_b)^2)
// and y the partner frequency of the channel.
__global__ void k_nodes_adj(Geo g, const double* __restrict__ w, const double* __restrict__ invh,
                            const double* __restrict__ gam, const double* __restrict__ dgam, double lam,
                            const double* __restrict__ nx, const double* __restrict__ ntw, const int* __restrict__ ncount,
                            const double* __restrict__ Wbar, double* __restrict__ gambar, double* __restrict__ dgbar) {
    const int id = blockIdx.x, ch = id / g.N, vi = id % g.N, N = g.N;
    const double v = w[vi];
    const double inv2pi = 1.0 / (2.0 * kPi);
    const double* X = nx + (size_t)id * g.nmax;
    const double* Wb = Wbar + (size_t)id * g.nmax;
    const int n = ncount[id];
    auto gg_adj = [&](double a, double b, double wbar) {
        if (wbar == 0.0) return;
        const double ga = a + interp_odd(w, invh, N, gam, a);
        const double gb = b + interp_odd(w, invh, N, gam, b);
        const double val = -1.0 / (ga * gb) * inv2pi;
        interp_odd_adj(w, invh, N, gambar, a, -wbar * val / ga);
        interp_odd_adj(w, invh, N, gambar, b, -wbar * val / gb);
    };
    if (threadIdx.x == 0) {
        for (int sg = 0; sg < 2; ++sg) {
            const double L = sg == 0 ? lam : -lam;
            if (ch == 0) {
                const double a = v - L;
                if (fabs(a) - lam >= 0.0) gg_adj(a, L, Wb[2 * sg] + Wb[2 * sg + 1]);
            } else if (ch == 1) {
                double a = v + L;
                if (fabs(a) - lam >= 0.0) gg_adj(a, L, Wb[2 * sg]);
                a = L - v;
                if (fabs(a) - lam >= 0.0) gg_adj(a, L, Wb[2 * sg + 1]);
            } else {
                double a = L - v;
                if (fabs(a) - lam >= 0.0) gg_adj(a, L, Wb[2 * sg]);
                a = v + L;
                if (fabs(a) - lam >= 0.0) gg_adj(a, L, Wb[2 * sg + 1]);
            }
        }
    }
    for (int k = 4 + threadIdx.x; k < n; k += blockDim.x) {
        const double pbar = Wb[k] * ntw[(size_t)id * g.nmax + k] * inv2pi;
        if (pbar == 0.0) continue;
        const double a = X[k];
        const double b = ch == 0 ? v - a : (ch == 1 ? a - v : v + a);
        const double ga = a + interp_odd(w, invh, N, gam, a);
        const double gb = b + interp_odd(w, invh, N, gam, b);
        const double da = interp_odd(w, invh, N, dgam, a);
        const double db = interp_odd(w, invh, N, dgam, b);
        const double tab = -db / (ga * gb * gb), tba = -da / (gb * ga * ga);
        interp_odd_adj(w, invh, N, gambar, a, pbar * (-tab - 2.0 * tba) / ga);
        interp_odd_adj(w, invh, N, gambar, b, pbar * (-2.0 * tab - tba) / gb);
        interp_odd_adj(w, invh, N, dgbar, b, -pbar / (ga * gb * gb));
        interp_odd_adj(w, invh, N, dgbar, a, -pbar / (gb * ga * ga));
    }
}

// Self-energy: dgamma_n = -(1/2pi) [H(+L) / (L + gamma(L)) + H(-L) / (-L + gamma(-L))] with H
// linear in Gamma; dgbar holds the full adjoint of dgamma (direct + through the node weights).
__global__ void k_sigma_adj(Geo g, Tabs tb, const double* __restrict__ w, const double* __restrict__ gam,
                            const double* __restrict__ G, double lam, const double* __restrict__ dgbar,
                            double* __restrict__ gambar, double* __restrict__ Gbar) {
    __shared__ double red[2 * 32];
    __shared__ double Hb[2];
    const int n = blockIdx.x;
    const double w1 = w[n];
    double H[2] = {0.0, 0.0};
    for (int sg = 0; sg < 2; ++sg) {
        const double w2 = sg == 0 ? lam : -lam;
        Desc<double> d;
        make_desc(w1 + w2, 0.0, w1 - w2, 1, 0, tb, g, d);
        double h = 0.0;
        for (int r = threadIdx.x; r < g.Ns; r += blockDim.x) h += (double)tb.mult[r] * row_value(G, d, tb, g, r, 0);
        h = 2.0 * h;
        if (threadIdx.x == 0) {
            Desc<double> e;
            make_desc(w1 + w2, w2 - w1, 0.0, 2, 0, tb, g, e);
            double f = 0.0;
            if (g.nc == 2) f = row_value(G, e, tb, g, 0, 0) + 3.0 * row_value(G, e, tb, g, 0, 1);
            else for (int c = 0; c < 4; ++c) f += row_value(G, e, tb, g, 0, c);
            h -= f;
        }
        H[sg] = h;
    }
    block_sum<double, 2>(H, red);
    if (threadIdx.x == 0) {
        const double db = dgbar[n];
        const double gp = lam + interp_odd(w, tb.invh, g.N, gam, lam);
        const double gm = -lam + interp_odd(w, tb.invh, g.N, gam, -lam);
        const double c = db / (2.0 * kPi);
        Hb[0] = -c / gp;
        Hb[1] = -c / gm;
        interp_odd_adj(w, tb.invh, g.N, gambar, lam, c * H[0] / (gp * gp));
        interp_odd_adj(w, tb.invh, g.N, gambar, -lam, c * H[1] / (gm * gm));
    }
    __syncthreads();
    for (int sg = 0; sg < 2; ++sg) {
        const double w2 = sg == 0 ? lam : -lam;
        const double hb = Hb[sg];
        Desc<double> d;
        make_desc(w1 + w2, 0.0, w1 - w2, 1, 0, tb, g, d);
        for (int r = threadIdx.x; r < g.Ns; r += blockDim.x) row_value_adj(Gbar, d, tb, g, r, 0, 2.0 * tb.mult[r] * hb);
        if (threadIdx.x == 0) {
            Desc<double> e;
            make_desc(w1 + w2, w2 - w1, 0.0, 2, 0, tb, g, e);
            if (g.nc == 2) {
                row_value_adj(Gbar, e, tb, g, 0, 0, -hb);
                row_value_adj(Gbar, e, tb, g, 0, 1, -3.0 * hb);
            } else {
                for (int c = 0; c < 4; ++c) row_value_adj(Gbar, e, tb, g, 0, c, -hb);
            }
        }
    }
}

// chi(k) = (1/N_b) sum_p cos(k . dr_p) sp_p  =>  adjoint of the pair correlations.
__global__ void k_chik_adj(int nk, const double* __restrict__ kp, const double* __restrict__ chik_bar,
                           const double* __restrict__ dr, int npairs, int nb, int nc, double* __restrict__ chibar) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    double a = 0.0;
    for (int i = 0; i < nk; ++i)
        a += chik_bar[i] * cos(kp[3 * i] * dr[3 * p] + kp[3 * i + 1] * dr[3 * p + 1] + kp[3 * i + 2] * dr[3 * p + 2]);
    a /= (double)nb;
    if (nc == 2) {
        chibar[(size_t)p * 2] = 0.0;
        chibar[(size_t)p * 2 + 1] = 3.0 * a;
    } else {
        chibar[(size_t)p * 4] = 0.0;
        for (int c = 1; c < 4; ++c) chibar[(size_t)p * 4 + c] = a;
    }
}

// Pair correlations (k_chi): chi_mu = [on] bub / 2pi - acc_mu / 16pi^2 with
// acc_mu = sum_{p,q} Wn_p Wn_q F_mu(p, q), bub = sum_k Wn_k, Wn(gamma) the exact segment weights.
template <int NC>
__global__ void k_chi_adj(Geo g, Tabs tb, const double* __restrict__ w, const double* __restrict__ gam,
                          const double* __restrict__ G, double lam, const int2* __restrict__ cmap,
                          const int* __restrict__ onsite, int ntot, const double* __restrict__ chibar,
                          double* __restrict__ gambar, double* __restrict__ Gbar) {
    __shared__ double y[kMaxFreq + 1];
    __shared__ double Wn[kMaxFreq + 1];
    __shared__ double Wnb[kMaxFreq + 1];
    __shared__ int Ksh;
    const int pidx = blockIdx.x;
    const int b = pidx / ntot;
    const int on = onsite[pidx];
    const int2 pm = cmap[pidx];
    const int2 pon = cmap[b * ntot + 0];
    const int N = g.N;
    double ab[NC];
#pragma unroll
    for (int mu = 0; mu < NC; ++mu) ab[mu] = -chibar[(size_t)pidx * NC + mu] / (16.0 * kPi * kPi);
    double bubbar = 0.0;
    if (on)
        for (int mu = 0; mu < NC; ++mu) bubbar += chibar[(size_t)pidx * NC + mu];
    bubbar /= 2.0 * kPi;
    if (threadIdx.x == 0) {
        int K = 0;
        y[K++] = lam;
        for (int i = 0; i < N; ++i) if (w[i] > lam) y[K++] = w[i];
        for (int k = 0; k < K; ++k) Wn[k] = 0.0;
        for (int k = 0; k + 1 < K; ++k) {
            const double ya = y[k] + interp_odd(w, tb.invh, N, gam, y[k]);
            const double yb = y[k + 1] + interp_odd(w, tb.invh, N, gam, y[k + 1]);
            const double seg = (y[k + 1] - y[k]) / (ya * yb);
            Wn[k] += 0.5 * seg;
            Wn[k + 1] += 0.5 * seg;
        }
        Wn[K - 1] += 1.0 / (y[K - 1] + interp_odd(w, tb.invh, N, gam, y[K - 1]));
        for (int k = 0; k < K; ++k) Wnb[k] = bubbar;
        Ksh = K;
    }
    __syncthreads();
    const int K = Ksh, M = 2 * K;
    for (int idx = threadIdx.x; idx < M * M; idx += blockDim.x) {
        const int pi = idx / M, qi = idx % M;
        const double xp = pi < K ? y[pi] : -y[pi - K];
        const double xq = qi < K ? y[qi] : -y[qi - K];
        const double wp = Wn[pi % K], wq = Wn[qi % K], wpq = wp * wq;
        Desc<double> d, de;
        make_desc(xp + xq, 0.0, xp - xq, 1, 0, tb, g, d);
        double v[NC], e[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = row_value(G, d, tb, g, pm.x, perm_of(pm.y, c));
        if (on) {
            make_desc(xp + xq, xq - xp, 0.0, 2, 0, tb, g, de);
#pragma unroll
            for (int c = 0; c < NC; ++c) e[c] = row_value(G, de, tb, g, pon.x, perm_of(pon.y, c));
        }
        double fsum = 0.0;
        double eb[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) eb[k] = 0.0;
#pragma unroll
        for (int mu = 0; mu < NC; ++mu) {
            double F = 4.0 * v[mu];
            if (on) {
                double x;
                if (NC == 2) x = mu == 0 ? 2.0 * (e[0] + 3.0 * e[1]) : 2.0 * (e[0] - e[1]);
                else {
                    x = 0.0;
                    for (int k = 0; k < 4; ++k) x += (mu == 0 || k == 0 || k == mu) ? 2.0 * e[k] : -2.0 * e[k];
                }
                F -= x;
                // dF_mu / d e_k = -dx_mu / d e_k
                if (NC == 2) {
                    eb[0] -= ab[mu] * wpq * 2.0;
                    eb[1] -= ab[mu] * wpq * (mu == 0 ? 6.0 : -2.0);
                } else {
                    for (int k = 0; k < 4; ++k) eb[k] -= ab[mu] * wpq * ((mu == 0 || k == 0 || k == mu) ? 2.0 : -2.0);
                }
            }
            fsum += ab[mu] * F;
            row_value_adj(Gbar, d, tb, g, pm.x, perm_of(pm.y, mu), 4.0 * wpq * ab[mu]);
        }
        if (on)
#pragma unroll
            for (int k = 0; k < NC; ++k) row_value_adj(Gbar, de, tb, g, pon.x, perm_of(pon.y, k), eb[k]);
        if (fsum != 0.0) {
            atomicAdd(&Wnb[pi % K], fsum * wq);
            atomicAdd(&Wnb[qi % K], fsum * wp);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k + 1 < K; ++k) {
            const double ya = y[k] + interp_odd(w, tb.invh, N, gam, y[k]);
            const double yb = y[k + 1] + interp_odd(w, tb.invh, N, gam, y[k + 1]);
            const double seg = (y[k + 1] - y[k]) / (ya * yb);
            const double sb = 0.5 * (Wnb[k] + Wnb[k + 1]);
            interp_odd_adj(w, tb.invh, N, gambar, y[k], -sb * seg / ya);
            interp_odd_adj(w, tb.invh, N, gambar, y[k + 1], -sb * seg / yb);
        }
        const double yt = y[K - 1] + interp_odd(w, tb.invh, N, gam, y[K - 1]);
        interp_odd_adj(w, tb.invh, N, gambar, y[K - 1], -Wnb[K - 1] / (yt * yt));
    }
}

// out = a - h b (the Euler step's transpose: ybar_n = ybar_n+1 - dLambda J^T ybar_n+1).
__global__ void k_axmy(long n, const double* a, const double* b, double h, double* out) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] - h * b[i];
}

}  // namespace
