// Reverse-mode (adjoint) kernels of the TRI core: the vector-Jacobian products of its
// self-energy flow, vertex flow and correlation measurement, in the three stages of the SU2 /
// XYZ adjoint (adjoint.cuh): the vertex part gives Gammabar and the adjoint of the node weights,
// k_nodes_adj carries the latter to gammabar and dgammabar, the self-energy part closes the
// chain.  Equations as in tri.cuh (Sec. 3, Eqs. frg:flowexplicit:1particle and
// frg:flowexplicit:2particle in the TRI parametrization; Eq. frg:correlation), differentiated
// term by term; transposed lookups scatter with FP64 atomics, so sums form in a run-dependent
// order.  Included by flow.cu after tri.cuh and adjoint.cuh.
#pragma once

namespace {

// Transpose of tri_value: scatter vbar = d/d(component c of the pair (ref, rep_r)) onto the
// stored corners, through the same site exchange, component map and signs.
__device__ __forceinline__ void tri_value_adj(double* __restrict__ Gbar, const Desc<double>& d, bool mneg, const Tabs& tb,
                                              const TabsT& tt, const Geo& g, int r, int c, double vbar) {
    if (vbar == 0.0) return;
    int rs = r, m = c;
    if (d.swap) { rs = tb.swap_r[r]; m = tt.swap_map[c * g.Ns + r]; }
    const int cs = m & 15;
    double* base = Gbar + cs * g.Ns + rs;
    const double* wgt = (cs & 3) == 0 ? d.wd : d.ws;
    const bool neg = ((m & 16) != 0) != (mneg && tri_mixed(c));
    const double v = neg ? -vbar : vbar;
    for (int k = 0; k < d.n; ++k)
        if (wgt[k] != 0.0) atomicAdd(base + d.off[k], wgt[k] * v);
}

struct AdjShT {
    Desc<double>* desc;   // kQTri * 4, without node weights
    int* mneg;            // kQTri * 4
    double* rows;         // kQTri * 2 * 16 Ns: raw rows A, B (slot tri_slot(r, c))
    double* rbar;         // their adjoints
    double* onrow;        // kQTri * 2 * 16: raw on-site rows C, D
    double* onbar;
    double* wq;           // kQTri: node weights
    double* wb;           // kQTri: adjoint of the node weights
    double* ob;           // 16 Ns: fbar of this triple, index r * 16 + c
};

__host__ __device__ inline size_t tri_adj_smem_bytes(int Ns) {
    auto rnd = [](size_t b) { return (b + 15) & ~size_t(15); };
    const size_t row = (size_t)Ns * 16;
    return rnd(sizeof(Desc<double>) * kQTri * 4) + rnd(sizeof(int) * kQTri * 4) + 2 * rnd(sizeof(double) * kQTri * 2 * row) +
           2 * rnd(sizeof(double) * kQTri * 2 * 16) + 2 * rnd(sizeof(double) * kQTri) + rnd(sizeof(double) * row);
}

// Vertex part: one CTA per stored (s, u, t) triple, the node loop of k_gamma_rhs_tri<double> on
// raw rows (the node weight W applied here): with fbar o of the triple's 16 N_s outputs,
//   s / u channel  out^{mu nu} += W sum_{x y} cf A^{xy} B^{(x^mu)(y^nu)}
//   t channel      out^{mu nu} += W [sum c2 A^{mu l} C'^{m (m^l^nu)} + sum c3 D^{(mu^l^m) l} B^{m nu}]
//                  out_o      -= 2 W sum_{signed products of o} A B (lattice sum)
// give Abar, Bbar, C'bar, Dbar (each carrying W) and Wbar (the bracket contracted with o).
__global__ void __launch_bounds__(kThreads) k_gamma_adj_tri(Geo g, Tabs tb, TabsT tt, const double* __restrict__ w,
                                                            const double* __restrict__ G, const double* __restrict__ nx,
                                                            const double* __restrict__ nW, const int* __restrict__ ncount,
                                                            const double* __restrict__ fbar, double* __restrict__ Gbar,
                                                            double* __restrict__ Wbar) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int row = g.Ns * 16;
    AdjShT sh;
    {
        size_t off = 0;
        auto take = [&](size_t bytes) { unsigned char* q = smem + off; off += (bytes + 15) & ~size_t(15); return q; };
        sh.desc = (Desc<double>*)take(sizeof(Desc<double>) * kQTri * 4);
        sh.mneg = (int*)take(sizeof(int) * kQTri * 4);
        sh.rows = (double*)take(sizeof(double) * kQTri * 2 * row);
        sh.rbar = (double*)take(sizeof(double) * kQTri * 2 * row);
        sh.onrow = (double*)take(sizeof(double) * kQTri * 2 * 16);
        sh.onbar = (double*)take(sizeof(double) * kQTri * 2 * 16);
        sh.wq = (double*)take(sizeof(double) * kQTri);
        sh.wb = (double*)take(sizeof(double) * kQTri);
        sh.ob = (double*)take(sizeof(double) * row);
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
    for (int o = tid; o < row; o += blockDim.x)
        sh.ob[o] = fbar[((size_t)(p * g.N + ti) * 16 + (o & 15)) * g.Ns + (o >> 4)];

    for (int ch = 0; ch < 3; ++ch) {
        const int vi = ch == 0 ? si : (ch == 1 ? ti : ui);
        const int cidx = ch * g.N + vi;
        const int nq = ncount[cidx];
        const double* X = nx + (size_t)cidx * g.nmax;
        const double* Wp = nW + (size_t)cidx * g.nmax;
        const int nrow = ch == 1 ? 4 : 2;
        for (int q0 = 0; q0 < nq; q0 += kQTri) {
            const int qn = min(kQTri, nq - q0);
            __syncthreads();
            for (int idx = tid; idx < qn * nrow; idx += blockDim.x) {
                const int q = idx / nrow, rw = idx % nrow;
                const double x = X[q0 + q];
                double a, b, c;
                node_args(ch, rw, x, s, t, u, w1p, w2p, w1, w2, a, b, c);
                const int exs = ch == 0 ? 0 : (ch == 2 ? 2 : (rw < 2 ? 1 : 2));
                make_desc(a, b, c, exs, vi, tb, g, sh.desc[q * 4 + rw]);
                sh.mneg[q * 4 + rw] = (b < 0.0) != (c < 0.0);
                if (rw == 0) { sh.wq[q] = Wp[q0 + q]; sh.wb[q] = 0.0; }
            }
            for (int j = tid; j < qn * 2 * row; j += blockDim.x) sh.rbar[j] = 0.0;
            for (int j = tid; j < qn * 2 * 16; j += blockDim.x) sh.onbar[j] = 0.0;
            __syncthreads();
            for (int idx = tid; idx < qn * 2 * row; idx += blockDim.x) {
                const int q = idx / (2 * row), rem = idx % (2 * row), rw = rem / row, e = rem % row;
                const int r = e >> 4, c = e & 15;
                sh.rows[(q * 2 + rw) * row + tri_slot(r, c)] =
                    tri_value<double>(G, sh.desc[q * 4 + rw], sh.mneg[q * 4 + rw] != 0, tb, tt, g, r, c);
            }
            if (ch == 1)
                for (int j = tid; j < qn * 2 * 16; j += blockDim.x) {
                    const int q = j / 32, rr = (j / 16) % 2, c = j % 16;
                    sh.onrow[j] = tri_value<double>(G, sh.desc[q * 4 + 2 + rr], sh.mneg[q * 4 + 2 + rr] != 0, tb, tt, g, 0, c);
                }
            __syncthreads();
            // site-local products, item (node q, site r)
            for (int item = tid; item < qn * g.Ns; item += blockDim.x) {
                const int q = item / g.Ns, r = item % g.Ns, sw = r & 15;
                const double W = sh.wq[q];
                const double* o = sh.ob + r * 16;
                const double* A = sh.rows + (q * 2) * row + r * 16;
                const double* B = A + row;
                double a[16], b[16], ab[16], bb[16];
                for (int k = 0; k < 16; ++k) { a[k] = A[k ^ sw]; b[k] = B[k ^ sw]; ab[k] = 0.0; bb[k] = 0.0; }
                double wsum = 0.0;
                if (ch != 1) {
                    for (int mu = 0; mu < 4; ++mu)
                        for (int nu = 0; nu < 4; ++nu)
                            for (int x = 0; x < 4; ++x)
                                for (int y = 0; y < 4; ++y) {
                                    const int cf = ch == 0 ? sr::tri::coef_s(mu, nu, x, y) : sr::tri::coef_u(mu, nu, x, y);
                                    const double ov = cf > 0 ? o[mu * 4 + nu] : -o[mu * 4 + nu];
                                    const int ka = x * 4 + y, kb = (x ^ mu) * 4 + (y ^ nu);
                                    ab[ka] += ov * b[kb];
                                    bb[kb] += ov * a[ka];
                                    wsum += ov * a[ka] * b[kb];
                                }
                } else {
                    const double* C0 = sh.onrow + (q * 2) * 16;
                    const double* D = sh.onrow + (q * 2 + 1) * 16;
                    double cp[16], cpb[16], db[16];
                    for (int k = 0; k < 16; ++k) {
                        const int mk = tt.onsite_map[r * 16 + k];
                        cp[k] = (mk & 16) ? -C0[mk & 15] : C0[mk & 15];
                        cpb[k] = 0.0;
                        db[k] = 0.0;
                    }
                    for (int mu = 0; mu < 4; ++mu)
                        for (int nu = 0; nu < 4; ++nu)
                            for (int l = 0; l < 4; ++l)
                                for (int m = 0; m < 4; ++m) {
                                    const double ov = o[mu * 4 + nu];
                                    const double o2 = sr::tri::coef_o2(mu, nu, l, m) > 0 ? ov : -ov;
                                    const double o3 = sr::tri::coef_o3(mu, nu, l, m) > 0 ? ov : -ov;
                                    const int ka = mu * 4 + l, kc = m * 4 + (m ^ l ^ nu);
                                    const int kd = (mu ^ l ^ m) * 4 + l, kb = m * 4 + nu;
                                    ab[ka] += o2 * cp[kc];
                                    cpb[kc] += o2 * a[ka];
                                    db[kd] += o3 * b[kb];
                                    bb[kb] += o3 * D[kd];
                                    wsum += o2 * a[ka] * cp[kc] + o3 * D[kd] * b[kb];
                                }
                    for (int k = 0; k < 16; ++k) {
                        const int mk = tt.onsite_map[r * 16 + k];
                        if (cpb[k] != 0.0) atomicAdd(&sh.onbar[(q * 2) * 16 + (mk & 15)], W * ((mk & 16) ? -cpb[k] : cpb[k]));
                        if (db[k] != 0.0) atomicAdd(&sh.onbar[(q * 2 + 1) * 16 + k], W * db[k]);
                    }
                }
                for (int k = 0; k < 16; ++k) {
                    if (ab[k] != 0.0) atomicAdd(&sh.rbar[(q * 2) * row + r * 16 + (k ^ sw)], W * ab[k]);
                    if (bb[k] != 0.0) atomicAdd(&sh.rbar[(q * 2 + 1) * row + r * 16 + (k ^ sw)], W * bb[k]);
                }
                if (wsum != 0.0) atomicAdd(&sh.wb[q], wsum);
            }
            // lattice sum: out_o -= 2 sum_q W_q sum_{products of o} sign A B
            if (ch == 1)
                for (int o = tid; o < row; o += blockDim.x) {
                    const double obv = sh.ob[o];
                    if (obv == 0.0) continue;
                    double wl[kQTri];
                    for (int q = 0; q < kQTri; ++q) wl[q] = 0.0;
                    for (int k = tt.lat_off[o]; k < tt.lat_off[o + 1]; ++k) {
                        const int2 en = tt.lat_ent[k];
                        const int ia = en.x, ib = en.y < 0 ? ~en.y : en.y;
                        const double cv = (en.y < 0 ? 2.0 : -2.0) * obv;
                        for (int q = 0; q < qn; ++q) {
                            const double W = sh.wq[q];
                            const double* Aq = sh.rows + (q * 2) * row;
                            const double* Bq = Aq + row;
                            atomicAdd(&sh.rbar[(q * 2) * row + ia], W * cv * Bq[ib]);
                            atomicAdd(&sh.rbar[(q * 2 + 1) * row + ib], W * cv * Aq[ia]);
                            wl[q] += cv * Aq[ia] * Bq[ib];
                        }
                    }
                    for (int q = 0; q < qn; ++q)
                        if (wl[q] != 0.0) atomicAdd(&sh.wb[q], wl[q]);
                }
            __syncthreads();
            for (int idx = tid; idx < qn * 2 * row; idx += blockDim.x) {
                const int q = idx / (2 * row), rem = idx % (2 * row), rw = rem / row, e = rem % row;
                const int r = e >> 4, c = e & 15;
                tri_value_adj(Gbar, sh.desc[q * 4 + rw], sh.mneg[q * 4 + rw] != 0, tb, tt, g, r, c,
                              sh.rbar[(q * 2 + rw) * row + tri_slot(r, c)]);
            }
            if (ch == 1)
                for (int j = tid; j < qn * 2 * 16; j += blockDim.x) {
                    const int q = j / 32, rr = (j / 16) % 2, c = j % 16;
                    tri_value_adj(Gbar, sh.desc[q * 4 + 2 + rr], sh.mneg[q * 4 + 2 + rr] != 0, tb, tt, g, 0, c, sh.onbar[j]);
                }
            for (int q = tid; q < qn; q += blockDim.x)
                if (sh.wb[q] != 0.0) atomicAdd(&Wbar[(size_t)cidx * g.nmax + q0 + q], sh.wb[q]);
        }
    }
}

// Self-energy (spin trace, as k_sigma_rhs_tri): dgamma_n = -(1/2pi) [H(+L) / (L + gamma(L)) +
// H(-L) / (-L + gamma(-L))] with H = 2 sum_j Gamma^00_{ref j} - sum_k Gamma^kk_{ref ref}, linear
// in Gamma; dgbar holds the full adjoint of dgamma.
__global__ void k_sigma_adj_tri(Geo g, Tabs tb, TabsT tt, const double* __restrict__ w, const double* __restrict__ gam,
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
        const bool mn = (w1 - w2) < 0.0;
        double h = 0.0;
        for (int r = threadIdx.x; r < g.Ns; r += blockDim.x) h += (double)tb.mult[r] * tri_value(G, d, mn, tb, tt, g, r, 0);
        h = 2.0 * h;
        if (threadIdx.x == 0) {
            Desc<double> e;
            make_desc(w1 + w2, w2 - w1, 0.0, 2, 0, tb, g, e);
            const bool me = (w2 - w1) < 0.0;
            double f = 0.0;
            for (int k = 0; k < 4; ++k) f += tri_value(G, e, me, tb, tt, g, 0, 5 * k);
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
        const bool mn = (w1 - w2) < 0.0;
        for (int r = threadIdx.x; r < g.Ns; r += blockDim.x) tri_value_adj(Gbar, d, mn, tb, tt, g, r, 0, 2.0 * tb.mult[r] * hb);
        if (threadIdx.x == 0) {
            Desc<double> e;
            make_desc(w1 + w2, w2 - w1, 0.0, 2, 0, tb, g, e);
            const bool me = (w2 - w1) < 0.0;
            for (int k = 0; k < 4; ++k) tri_value_adj(Gbar, e, me, tb, tt, g, 0, 5 * k, -hb);
        }
    }
}

// chi(k) = (1/N_b) sum_p cos(k . dr_p) (chi^xx + chi^yy + chi^zz)_p  =>  adjoint of the pair
// correlations (components 5, 10, 15).
__global__ void k_chik_adj_tri(int nk, const double* __restrict__ kp, const double* __restrict__ chik_bar,
                               const double* __restrict__ dr, int npairs, int nb, double* __restrict__ chibar) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    double a = 0.0;
    for (int i = 0; i < nk; ++i)
        a += chik_bar[i] * cos(kp[3 * i] * dr[3 * p] + kp[3 * i + 1] * dr[3 * p + 1] + kp[3 * i + 2] * dr[3 * p + 2]);
    a /= (double)nb;
    for (int c = 0; c < 16; ++c) chibar[(size_t)p * 16 + c] = (c == 5 || c == 10 || c == 15) ? a : 0.0;
}

// Pair correlations of the TRI core (k_chi_tri): chi^c = [on, c diagonal] bub / 2pi -
// acc^c / 16pi^2 with acc^c = sum_{p,q} Wn_p Wn_q F^c(p, q), F^{mu nu} = 4 v^{mu nu} - [on]
// sum_l (+-2) e^{(mu^nu^l) l}.
__global__ void k_chi_adj_tri(Geo g, Tabs tb, TabsT tt, const double* __restrict__ w, const double* __restrict__ gam,
                              const double* __restrict__ G, double lam, const int* __restrict__ cr, const int* __restrict__ cm,
                              const int* __restrict__ onsite, int ntot, const double* __restrict__ chibar,
                              double* __restrict__ gambar, double* __restrict__ Gbar) {
    __shared__ double y[kMaxFreq + 1];
    __shared__ double Wn[kMaxFreq + 1];
    __shared__ double Wnb[kMaxFreq + 1];
    __shared__ int Ksh;
    const int pidx = blockIdx.x;
    const int b = pidx / ntot;
    const int on = onsite[pidx];
    const int r = cr[pidx];
    const int r0 = cr[b * ntot];
    const int* m = cm + (size_t)pidx * 16;
    const int* m0 = cm + (size_t)b * ntot * 16;
    const int N = g.N;
    double ab[16];
    for (int c = 0; c < 16; ++c) ab[c] = -chibar[(size_t)pidx * 16 + c] / (16.0 * kPi * kPi);
    double bubbar = 0.0;
    if (on)
        for (int c = 0; c < 16; c += 5) bubbar += chibar[(size_t)pidx * 16 + c];
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
        const bool mn = (xp - xq) < 0.0;
        double v[16], e[16], eb[16];
        for (int c = 0; c < 16; ++c) {
            const int mc = m[c];
            const double x = tri_value(G, d, mn, tb, tt, g, r, mc & 15);
            v[c] = (mc & 16) ? -x : x;
            eb[c] = 0.0;
        }
        bool me = false;
        if (on) {
            make_desc(xp + xq, xq - xp, 0.0, 2, 0, tb, g, de);
            me = (xq - xp) < 0.0;
            for (int c = 0; c < 16; ++c) {
                const int mc = m0[c];
                const double x = tri_value(G, de, me, tb, tt, g, r0, mc & 15);
                e[c] = (mc & 16) ? -x : x;
            }
        }
        double fsum = 0.0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu) {
                const int c = mu * 4 + nu;
                double F = 4.0 * v[c];
                if (on)
                    for (int l = 0; l < 4; ++l) {
                        const int k = (mu ^ nu ^ l) * 4 + l;
                        const double cx = sr::tri::coef_x(mu, nu, l) > 0 ? 2.0 : -2.0;
                        F -= cx * e[k];
                        eb[k] -= cx * wpq * ab[c];
                    }
                fsum += ab[c] * F;
                const int mc = m[c];
                tri_value_adj(Gbar, d, mn, tb, tt, g, r, mc & 15, ((mc & 16) ? -4.0 : 4.0) * wpq * ab[c]);
            }
        if (on)
            for (int k = 0; k < 16; ++k) {
                const int mc = m0[k];
                tri_value_adj(Gbar, de, me, tb, tt, g, r0, mc & 15, (mc & 16) ? -eb[k] : eb[k]);
            }
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

}  // namespace
