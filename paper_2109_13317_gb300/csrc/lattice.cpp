// Host-side lattice truncation and symmetry analysis (Sec. 4.1 of arXiv:2109.13317).
//
// The symmetry search works on the real-space representation of the lattice with the
// absolute precision eps of the paper (1e-5 by default): a candidate isometry
// x -> O x + c maps the primitive vectors onto lattice vectors with the same Gram matrix
// and the basis sites onto lattice sites; it is a symmetry of the model if it maps bonds
// onto bonds and couplings onto couplings up to one global permutation of the spin
// components x, y, z.  Symmetries are then applied in exact integer arithmetic.
#include "lattice.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>

namespace sr {

SiteKey Sym::apply(const SiteKey& s) const {
    SiteKey r;
    for (int i = 0; i < 3; ++i) r.n[i] = M[i][0] * s.n[0] + M[i][1] * s.n[1] + M[i][2] * s.n[2] + m[s.b][i];
    r.b = pb[s.b];
    return r;
}

namespace {

struct PairKey {
    int bi, bj, d0, d1, d2;
    bool operator<(const PairKey& o) const {
        if (bi != o.bi) return bi < o.bi;
        if (bj != o.bj) return bj < o.bj;
        if (d0 != o.d0) return d0 < o.d0;
        if (d1 != o.d1) return d1 < o.d1;
        return d2 < o.d2;
    }
};

struct Mat3 { double a[3][3]; };

bool invert3(const double m[3][3], double inv[3][3]) {
    double det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                 m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    if (std::fabs(det) < 1e-12) return false;
    inv[0][0] = (m[1][1] * m[2][2] - m[1][2] * m[2][1]) / det;
    inv[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) / det;
    inv[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) / det;
    inv[1][0] = (m[1][2] * m[2][0] - m[1][0] * m[2][2]) / det;
    inv[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) / det;
    inv[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) / det;
    inv[2][0] = (m[1][0] * m[2][1] - m[1][1] * m[2][0]) / det;
    inv[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) / det;
    inv[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) / det;
    return true;
}

const int kPerms[6][3] = {{1, 2, 3}, {1, 3, 2}, {2, 1, 3}, {2, 3, 1}, {3, 1, 2}, {3, 2, 1}};

}  // namespace

}  // namespace sr

void sr_lattice::position(const sr::SiteKey& s, double out[3]) const {
    for (int k = 0; k < 3; ++k)
        out[k] = s.n[0] * prim[0][k] + s.n[1] * prim[1][k] + s.n[2] * prim[2][k] + basis[3 * s.b + k];
}

sr::PairMap sr_lattice::map_pair(const sr::SiteKey& i1, const sr::SiteKey& i2) const {
    sr::SiteKey d;
    for (int k = 0; k < 3; ++k) d.n[k] = i2.n[k] - i1.n[k];
    d.b = i2.b;
    const sr::Sym& g = T[i1.b];
    sr::SiteKey j = g.apply(d);
    sr::PairMap pm;
    auto it = site_index.find(j);
    if (it == site_index.end()) { pm.r = -1; pm.perm = {0, 1, 2, 3}; return pm; }
    int idx = it->second;
    pm.r = site_r[idx];
    for (int c = 0; c < 4; ++c) pm.perm[c] = site_perm[idx][g.sp[c]];
    return pm;
}

sr::PairMap16 sr_lattice::map_pair16(const sr::SiteKey& i1, const sr::SiteKey& i2) const {
    sr::SiteKey d;
    for (int k = 0; k < 3; ++k) d.n[k] = i2.n[k] - i1.n[k];
    d.b = i2.b;
    const sr::Sym& g = T[i1.b];
    sr::SiteKey j = g.apply(d);
    sr::PairMap16 pm;
    auto it = site_index.find(j);
    if (it == site_index.end()) {
        pm.r = -1;
        for (int c = 0; c < 16; ++c) pm.m[c] = c;
        return pm;
    }
    const int idx = it->second;
    pm.r = site_r[idx];
    // Gamma^{mu nu}_{i1 i2} = sg(mu) sg(nu) Gamma^{sp(mu) sp(nu)}_{ref, j}, then the site map of j
    for (int c = 0; c < 16; ++c) {
        const int mu = c / 4, nu = c % 4;
        const int cj = g.sp[mu] * 4 + g.sp[nu];
        const int neg = (g.sg[mu] * g.sg[nu] < 0) ? 16 : 0;
        pm.m[c] = site_map16[idx][cj] ^ neg;
    }
    return pm;
}

namespace sr {

sr_status build_lattice(const sr_lattice_desc* d, sr_lattice* lat, std::string* msg) {
    const double eps = d->eps > 0 ? d->eps : 1e-5;
    lat->eps = eps;
    lat->nb = d->n_basis;
    lat->L = d->range_L;
    lat->backend = d->backend;
    lat->nc = d->backend == SR_SU2 ? 2 : (d->backend == SR_XYZ ? 4 : 16);
    std::memcpy(lat->prim, d->prim, sizeof(lat->prim));
    lat->basis.assign(d->basis_xyz, d->basis_xyz + 3 * d->n_basis);
    lat->bonds.assign(d->bonds, d->bonds + d->n_bonds);
    lat->couplings.assign(d->couplings, d->couplings + d->n_couplings);
    const int nb = lat->nb;

    // A: columns = primitive vectors
    double A[3][3], Ainv[3][3];
    for (int i = 0; i < 3; ++i) for (int k = 0; k < 3; ++k) A[k][i] = d->prim[i][k];
    if (!invert3(A, Ainv)) { *msg = "primitive vectors are linearly dependent"; return SR_EINVAL; }
    auto to_lattice = [&](const double x[3], int n[3]) -> bool {
        for (int i = 0; i < 3; ++i) {
            double v = Ainv[i][0] * x[0] + Ainv[i][1] * x[1] + Ainv[i][2] * x[2];
            double r = std::round(v);
            if (std::fabs(v - r) > eps) return false;
            n[i] = (int)r;
        }
        return true;
    };

    // bonds (both directions) and couplings J_{(0,bi),(dn,bj)} (reading: J_ij = M, J_ji = M^T)
    std::map<PairKey, int> bondset;
    for (const sr_bond& b : lat->bonds) {
        if (b.from_basis < 0 || b.from_basis >= nb || b.to_basis < 0 || b.to_basis >= nb) {
            *msg = "bond references a basis site out of range"; return SR_EINVAL;
        }
        bondset[{b.from_basis, b.to_basis, b.da[0], b.da[1], b.da[2]}] = 1;
        bondset[{b.to_basis, b.from_basis, -b.da[0], -b.da[1], -b.da[2]}] = 1;
    }
    std::map<PairKey, std::array<double, 9>> cmap;
    for (const sr_coupling& c : lat->couplings) {
        if (c.from[3] < 0 || c.from[3] >= nb || c.to[3] < 0 || c.to[3] >= nb) {
            *msg = "coupling references a basis site out of range"; return SR_EINVAL;
        }
        PairKey k1{c.from[3], c.to[3], c.to[0] - c.from[0], c.to[1] - c.from[1], c.to[2] - c.from[2]};
        PairKey k2{c.to[3], c.from[3], -k1.d0, -k1.d1, -k1.d2};
        auto& a = cmap[k1];
        auto& b = cmap[k2];
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) {
            a[3 * i + j] += c.M[i][j];
            b[3 * j + i] += c.M[i][j];
        }
    }
    // the chosen core must be able to represent the couplings
    for (auto& kv : cmap) {
        const auto& J = kv.second;
        if (lat->backend == SR_TRI) continue;
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j)
            if (i != j && std::fabs(J[3 * i + j]) > eps) {
                *msg = "off-diagonal couplings need the TRI core";
                return SR_EUNSUPPORTED;
            }
        if (lat->backend == SR_SU2 && (std::fabs(J[0] - J[4]) > eps || std::fabs(J[0] - J[8]) > eps)) {
            *msg = "the SU2 core needs Heisenberg couplings (J^xx = J^yy = J^zz)";
            return SR_EUNSUPPORTED;
        }
    }

    // candidate lattice vectors for the images of the primitive vectors
    double G[3][3];
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j)
        G[i][j] = d->prim[i][0] * d->prim[j][0] + d->prim[i][1] * d->prim[j][1] + d->prim[i][2] * d->prim[j][2];
    struct Cand { int n[3]; double v[3]; };
    std::vector<Cand> cands;
    const int R = 3;
    for (int a = -R; a <= R; ++a) for (int b = -R; b <= R; ++b) for (int c = -R; c <= R; ++c) {
        if (!a && !b && !c) continue;
        Cand cd{{a, b, c}, {0, 0, 0}};
        for (int k = 0; k < 3; ++k) cd.v[k] = a * d->prim[0][k] + b * d->prim[1][k] + c * d->prim[2][k];
        cands.push_back(cd);
    }
    auto dot = [](const double* x, const double* y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; };
    const double geps = eps * 10.0;

    lat->T.assign(nb, Sym());
    std::vector<bool> haveT(nb, false);
    lat->G0.clear();
    std::vector<int> perm_order;
    // candidate spin maps: SU2 the identity, XYZ the permutations of x, y, z, TRI the 24
    // proper rotations among the signed permutations
    struct SpinMap { int sp[3]; int sg[3]; };
    std::vector<SpinMap> spin_maps;
    if (lat->backend == SR_SU2) spin_maps.push_back({{1, 2, 3}, {1, 1, 1}});
    else if (lat->backend == SR_XYZ) {
        for (int p = 0; p < 6; ++p) spin_maps.push_back({{kPerms[p][0], kPerms[p][1], kPerms[p][2]}, {1, 1, 1}});
    } else {
        for (int p = 0; p < 6; ++p)
            for (int sm = 0; sm < 8; ++sm) {
                SpinMap q{{kPerms[p][0], kPerms[p][1], kPerms[p][2]}, {(sm & 1) ? -1 : 1, (sm & 2) ? -1 : 1, (sm & 4) ? -1 : 1}};
                // determinant of the signed permutation matrix: parity of the permutation times the signs
                int inv = 0;
                for (int a = 0; a < 3; ++a) for (int b = a + 1; b < 3; ++b) inv += q.sp[a] > q.sp[b];
                const int det = ((inv & 1) ? -1 : 1) * q.sg[0] * q.sg[1] * q.sg[2];
                if (det == 1) spin_maps.push_back(q);
            }
    }
    const int nperm = (int)spin_maps.size();

    for (const Cand& c0 : cands) {
        if (std::fabs(dot(c0.v, c0.v) - G[0][0]) > geps) continue;
        for (const Cand& c1 : cands) {
            if (std::fabs(dot(c1.v, c1.v) - G[1][1]) > geps || std::fabs(dot(c0.v, c1.v) - G[0][1]) > geps) continue;
            for (const Cand& c2 : cands) {
                if (std::fabs(dot(c2.v, c2.v) - G[2][2]) > geps || std::fabs(dot(c0.v, c2.v) - G[0][2]) > geps ||
                    std::fabs(dot(c1.v, c2.v) - G[1][2]) > geps) continue;
                // O = V A^{-1}, V columns = images of the primitive vectors
                double V[3][3], O[3][3];
                for (int k = 0; k < 3; ++k) { V[k][0] = c0.v[k]; V[k][1] = c1.v[k]; V[k][2] = c2.v[k]; }
                for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j)
                    O[i][j] = V[i][0] * Ainv[0][j] + V[i][1] * Ainv[1][j] + V[i][2] * Ainv[2][j];
                Sym g;
                for (int i = 0; i < 3; ++i) { g.M[i][0] = c0.n[i]; g.M[i][1] = c1.n[i]; g.M[i][2] = c2.n[i]; }
                for (int src = 0; src < nb; ++src) {
                    // x -> O x + c with O p_src + c = p_0
                    double cvec[3];
                    for (int k = 0; k < 3; ++k)
                        cvec[k] = lat->basis[k] - (O[k][0] * lat->basis[3 * src] + O[k][1] * lat->basis[3 * src + 1] +
                                                   O[k][2] * lat->basis[3 * src + 2]);
                    g.m.assign(nb, {0, 0, 0});
                    g.pb.assign(nb, -1);
                    bool ok = true;
                    std::vector<bool> used(nb, false);
                    for (int bp = 0; bp < nb && ok; ++bp) {
                        double y[3];
                        for (int k = 0; k < 3; ++k)
                            y[k] = O[k][0] * lat->basis[3 * bp] + O[k][1] * lat->basis[3 * bp + 1] +
                                   O[k][2] * lat->basis[3 * bp + 2] + cvec[k];
                        int found = -1;
                        for (int bq = 0; bq < nb; ++bq) {
                            double x[3] = {y[0] - lat->basis[3 * bq], y[1] - lat->basis[3 * bq + 1], y[2] - lat->basis[3 * bq + 2]};
                            int n[3];
                            if (to_lattice(x, n)) { found = bq; g.m[bp] = {n[0], n[1], n[2]}; break; }
                        }
                        if (found < 0 || used[found]) ok = false;
                        else { used[found] = true; g.pb[bp] = found; }
                    }
                    if (!ok) continue;
                    // bonds onto bonds
                    for (const sr_bond& b : lat->bonds) {
                        SiteKey s1{{0, 0, 0}, b.from_basis}, s2{{b.da[0], b.da[1], b.da[2]}, b.to_basis};
                        SiteKey t1 = g.apply(s1), t2 = g.apply(s2);
                        PairKey k{t1.b, t2.b, t2.n[0] - t1.n[0], t2.n[1] - t1.n[1], t2.n[2] - t1.n[2]};
                        if (!bondset.count(k)) { ok = false; break; }
                    }
                    if (!ok) continue;
                    // couplings onto couplings up to one spin permutation
                    int chosen = -1;
                    for (int p = 0; p < nperm && chosen < 0; ++p) {
                        const int* sp = spin_maps[p].sp;  // spin x,y,z -> sp[0], sp[1], sp[2] (1-based)
                        const int* sgn = spin_maps[p].sg;
                        bool good = true;
                        for (auto& kv : cmap) {
                            SiteKey s1{{0, 0, 0}, kv.first.bi}, s2{{kv.first.d0, kv.first.d1, kv.first.d2}, kv.first.bj};
                            SiteKey t1 = g.apply(s1), t2 = g.apply(s2);
                            PairKey k{t1.b, t2.b, t2.n[0] - t1.n[0], t2.n[1] - t1.n[1], t2.n[2] - t1.n[2]};
                            auto it = cmap.find(k);
                            for (int a = 0; a < 3 && good; ++a) for (int bb = 0; bb < 3 && good; ++bb) {
                                double Jimg = it == cmap.end() ? 0.0 : it->second[3 * (sp[a] - 1) + (sp[bb] - 1)];
                                if (std::fabs(Jimg - sgn[a] * sgn[bb] * kv.second[3 * a + bb]) > eps) good = false;
                            }
                            if (!good) break;
                        }
                        if (good) chosen = p;
                    }
                    if (chosen < 0) continue;
                    g.sp = {0, spin_maps[chosen].sp[0], spin_maps[chosen].sp[1], spin_maps[chosen].sp[2]};
                    g.sg = {1, spin_maps[chosen].sg[0], spin_maps[chosen].sg[1], spin_maps[chosen].sg[2]};
                    if (src == 0) lat->G0.push_back(g);
                    if (!haveT[src]) { lat->T[src] = g; haveT[src] = true; }
                }
            }
        }
    }
    // the reference site maps onto itself by the identity
    {
        Sym id;
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) id.M[i][j] = (i == j);
        id.m.assign(nb, {0, 0, 0});
        id.pb.resize(nb);
        for (int b = 0; b < nb; ++b) id.pb[b] = b;
        id.sp = {0, 1, 2, 3};
        lat->T[0] = id;
        haveT[0] = haveT[0] || !lat->G0.empty();
    }
    for (int b = 0; b < nb; ++b)
        if (!haveT[b]) {
            *msg = "basis site " + std::to_string(b) + " is not equivalent to basis site 0 under the model's symmetries";
            return SR_ESYMMETRY;
        }
    if (lat->G0.empty()) { *msg = "no identity symmetry found (eps too small?)"; return SR_ESYMMETRY; }

    // sites within bond distance L of the reference site, breadth-first
    auto bfs = [&](SiteKey start, std::vector<SiteKey>& out) {
        std::unordered_map<SiteKey, int, SiteKeyHash> depth;
        std::deque<SiteKey> q;
        depth[start] = 0;
        q.push_back(start);
        out.clear();
        while (!q.empty()) {
            SiteKey cur = q.front();
            q.pop_front();
            out.push_back(cur);
            int dc = depth[cur];
            if (dc >= lat->L) continue;
            for (const sr_bond& b : lat->bonds) {
                for (int dir = 0; dir < 2; ++dir) {
                    SiteKey nx;
                    if (dir == 0) {
                        if (cur.b != b.from_basis) continue;
                        nx.b = b.to_basis;
                        for (int k = 0; k < 3; ++k) nx.n[k] = cur.n[k] + b.da[k];
                    } else {
                        if (cur.b != b.to_basis) continue;
                        nx.b = b.from_basis;
                        for (int k = 0; k < 3; ++k) nx.n[k] = cur.n[k] - b.da[k];
                    }
                    if (depth.count(nx)) continue;
                    depth[nx] = dc + 1;
                    q.push_back(nx);
                }
            }
        }
    };
    bfs(SiteKey{{0, 0, 0}, 0}, lat->sites);
    const int ntot = (int)lat->sites.size();
    lat->Ntot = ntot;
    lat->site_index.clear();
    for (int i = 0; i < ntot; ++i) lat->site_index[lat->sites[i]] = i;

    // orbits of the point group: representative = first site of the orbit in BFS order
    lat->site_r.assign(ntot, -1);
    lat->site_perm.assign(ntot, Perm{0, 1, 2, 3});
    {
        Map16 id;
        for (int c = 0; c < 16; ++c) id[c] = c;
        lat->site_map16.assign(ntot, id);
    }
    lat->rep.clear();
    for (int i = 0; i < ntot; ++i) {
        if (lat->site_r[i] >= 0) continue;
        int r = (int)lat->rep.size();
        lat->rep.push_back(i);
        lat->site_r[i] = r;  // the representative itself: identity component map
        for (const Sym& g : lat->G0) {
            SiteKey j = g.apply(lat->sites[i]);
            auto it = lat->site_index.find(j);
            if (it == lat->site_index.end()) { *msg = "point group maps a site out of range"; return SR_ESYMMETRY; }
            int jj = it->second;
            if (lat->site_r[jj] >= 0) continue;
            lat->site_r[jj] = r;
            // Gamma^{c}_{ref, rep} = Gamma^{sp(c)}_{ref, j}  =>  component c' of (ref, j) is stored c = sp^{-1}(c')
            Perm inv{0, 0, 0, 0};
            for (int c = 0; c < 4; ++c) inv[g.sp[c]] = c;
            lat->site_perm[jj] = inv;
            // TRI: Gamma^{sp(mu) sp(nu)}_{ref, j} = sg(mu) sg(nu) Gamma^{mu nu}_{ref, rep}
            for (int c = 0; c < 16; ++c) {
                const int mu = inv[c / 4], nu = inv[c % 4];
                lat->site_map16[jj][c] = (mu * 4 + nu) | ((g.sg[mu] * g.sg[nu] < 0) ? 16 : 0);
            }
        }
    }
    lat->Ns = (int)lat->rep.size();
    if (lat->backend == SR_SU2)
        for (auto& p : lat->site_perm) p = Perm{0, 1, 2, 3};

    const int Ns = lat->Ns;
    lat->mult.assign(Ns, 0);
    for (int i = 0; i < ntot; ++i) lat->mult[lat->site_r[i]]++;

    SiteKey ref{{0, 0, 0}, 0};
    lat->swap_r.assign(Ns, 0);
    lat->swap_perm.assign(Ns, Perm{0, 1, 2, 3});
    lat->onsite_perm.assign(Ns, Perm{0, 1, 2, 3});
    lat->init_gamma.assign((size_t)Ns * lat->nc, 0.0);
    lat->swap_map16.clear();
    lat->onsite_map16.clear();
    for (int r = 0; r < Ns; ++r) {
        const SiteKey& s = lat->sites[lat->rep[r]];
        PairMap pm = lat->map_pair(s, ref);
        if (pm.r < 0) { *msg = "exchanged pair out of range"; return SR_ESYMMETRY; }
        lat->swap_r[r] = pm.r;
        lat->swap_perm[r] = pm.perm;
        PairMap po = lat->map_pair(s, s);
        if (po.r != 0) { *msg = "on-site pair does not map to the reference site"; return SR_ESYMMETRY; }
        lat->onsite_perm[r] = po.perm;
        if (lat->nc == 16) {
            const PairMap16 ps = lat->map_pair16(s, ref);
            const PairMap16 pq = lat->map_pair16(s, s);
            Map16 sw;
            for (int c = 0; c < 16; ++c) sw[c] = ps.m[(c % 4) * 4 + c / 4];   // exchanged pair: mu <-> nu
            lat->swap_map16.push_back(sw);
            lat->onsite_map16.push_back(pq.m);
        }
        auto it = cmap.find(PairKey{0, s.b, s.n[0], s.n[1], s.n[2]});
        if (it != cmap.end()) {
            if (lat->nc == 16) {
                for (int a = 1; a < 4; ++a)
                    for (int b = 1; b < 4; ++b) lat->init_gamma[(size_t)r * 16 + a * 4 + b] = it->second[3 * (a - 1) + (b - 1)] / 4.0;
            } else if (lat->nc == 2) {
                lat->init_gamma[(size_t)r * 2 + 1] = it->second[8] / 4.0;
            } else {
                for (int c = 1; c < 4; ++c) lat->init_gamma[(size_t)r * 4 + c] = it->second[4 * (c - 1)] / 4.0;
            }
        }
    }
    if (lat->backend == SR_SU2) {
        for (auto& p : lat->swap_perm) p = Perm{0, 1, 2, 3};
        for (auto& p : lat->onsite_perm) p = Perm{0, 1, 2, 3};
    }

    // lattice-sum table: for each output site r2 (pair (ref, rep_r2)), every j within range of
    // both the reference site and rep_r2, with the stored sites of (ref, j) and (j, rep_r2)
    lat->rpa_off.assign(Ns + 1, 0);
    lat->rpa.clear();
    lat->rpa16.clear();
    for (int r2 = 0; r2 < Ns; ++r2) {
        const SiteKey& i2 = lat->sites[lat->rep[r2]];
        for (int j = 0; j < ntot; ++j) {
            PairMap pb = lat->map_pair(lat->sites[j], i2);
            if (pb.r < 0) continue;
            RpaEntry e;
            e.rA = lat->site_r[j];
            e.pA = lat->site_perm[j];
            e.rB = pb.r;
            e.pB = pb.perm;
            if (lat->backend == SR_SU2) { e.pA = Perm{0, 1, 2, 3}; e.pB = Perm{0, 1, 2, 3}; }
            lat->rpa.push_back(e);
            if (lat->nc == 16) {
                RpaEntry16 e16;
                e16.rA = e.rA;
                e16.mA = lat->site_map16[j];
                PairMap16 pb16 = lat->map_pair16(lat->sites[j], i2);
                e16.rB = pb16.r;
                e16.mB = pb16.m;
                lat->rpa16.push_back(e16);
            }
        }
        lat->rpa_off[r2 + 1] = (int)lat->rpa.size();
    }

    // correlation sites: for each basis b the sites within range of (0, b)
    lat->chi_sites.clear();
    lat->chi_map.clear();
    lat->chi_map16.clear();
    lat->chi_dr.clear();
    lat->chi_onsite.clear();
    for (int b = 0; b < nb; ++b) {
        std::vector<SiteKey> lst;
        bfs(SiteKey{{0, 0, 0}, b}, lst);
        if ((int)lst.size() != ntot) { *msg = "basis sites have different neighbourhoods"; return SR_ESYMMETRY; }
        SiteKey sb{{0, 0, 0}, b};
        double pb[3];
        lat->position(sb, pb);
        for (const SiteKey& j : lst) {
            lat->chi_sites.push_back(j);
            PairMap pm = lat->map_pair(sb, j);
            if (pm.r < 0) { *msg = "correlation pair out of range"; return SR_ESYMMETRY; }
            if (lat->backend == SR_SU2) pm.perm = Perm{0, 1, 2, 3};
            lat->chi_map.push_back(pm);
            if (lat->nc == 16) lat->chi_map16.push_back(lat->map_pair16(sb, j));
            double pj[3];
            lat->position(j, pj);
            for (int k = 0; k < 3; ++k) lat->chi_dr.push_back(pb[k] - pj[k]);
            lat->chi_onsite.push_back(j == sb ? 1 : 0);
        }
    }
    return SR_OK;
}

}  // namespace sr

namespace sr {

namespace {
// Coupling matrix of the pair ((0, b1), (d, b2)) with the matrices Ms (per listed interaction):
// sum of M over interactions from the first site to the second and of M^T over the reverse.
std::array<double, 9> pair_coupling(const sr_lattice* lat, int b1, const SiteKey& j, const double* Ms) {
    std::array<double, 9> acc{};
    for (size_t c = 0; c < lat->couplings.size(); ++c) {
        const sr_coupling& cp = lat->couplings[c];
        const double* M = Ms + 9 * c;
        if (cp.from[3] == b1 && cp.to[3] == j.b && cp.to[0] - cp.from[0] == j.n[0] && cp.to[1] - cp.from[1] == j.n[1] &&
            cp.to[2] - cp.from[2] == j.n[2])
            for (int k = 0; k < 9; ++k) acc[k] += M[k];
        if (cp.to[3] == b1 && cp.from[3] == j.b && cp.from[0] - cp.to[0] == j.n[0] && cp.from[1] - cp.to[1] == j.n[1] &&
            cp.from[2] - cp.to[2] == j.n[2])
            for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) acc[3 * a + b] += M[3 * b + a];
    }
    return acc;
}
}  // namespace

sr_status tangent_init(const sr_lattice* lat, int npar, const double* dM, std::vector<double>* out, std::string* msg) {
    const int nc = lat->nc, Ns = lat->Ns;
    const size_t ncoup = lat->couplings.size();
    out->assign((size_t)Ns * nc * npar, 0.0);
    if (nc == 16) {
        // TRI: the initial vertex J_ab / 4 in the slots (a, b), a, b = x, y, z (as the flow's
        // own initial vertex), and every pair's derivative must be the signed image of its
        // stored pair under the pair's component map
        for (int p = 0; p < npar; ++p) {
            const double* Ms = dM + (size_t)p * ncoup * 9;
            for (int r = 0; r < Ns; ++r) {
                const auto J = pair_coupling(lat, 0, lat->sites[lat->rep[r]], Ms);
                for (int a = 1; a < 4; ++a)
                    for (int b = 1; b < 4; ++b) (*out)[((size_t)r * 16 + a * 4 + b) * npar + p] = J[3 * (a - 1) + (b - 1)] / 4.0;
            }
            for (size_t i = 0; i < lat->chi_sites.size(); ++i) {
                const int b = (int)(i / lat->Ntot);
                const SiteKey& j = lat->chi_sites[i];
                const auto J = pair_coupling(lat, b, SiteKey{{j.n[0], j.n[1], j.n[2]}, j.b}, Ms);
                const PairMap16& pm = lat->chi_map16[i];
                for (int c = 0; c < 16; ++c) {
                    const int mu = c / 4, nu = c % 4;
                    const double want = (mu > 0 && nu > 0) ? J[3 * (mu - 1) + (nu - 1)] / 4.0 : 0.0;
                    const int m = pm.m[c];
                    const double img = (*out)[((size_t)pm.r * 16 + (m & 15)) * npar + p] * ((m & 16) ? -1.0 : 1.0);
                    if (std::fabs(want - img) > lat->eps) {
                        *msg = "tangent direction " + std::to_string(p) + " breaks a symmetry used to reduce the lattice";
                        return SR_ESYMMETRY;
                    }
                }
            }
        }
        return SR_OK;
    }
    for (int p = 0; p < npar; ++p) {
        const double* Ms = dM + (size_t)p * ncoup * 9;
        std::vector<std::array<double, 9>> rep(Ns);
        for (int r = 0; r < Ns; ++r) rep[r] = pair_coupling(lat, 0, lat->sites[lat->rep[r]], Ms);
        for (int r = 0; r < Ns; ++r) {
            const auto& J = rep[r];
            for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b)
                if (a != b && std::fabs(J[3 * a + b]) > lat->eps) { *msg = "tangent direction has off-diagonal couplings"; return SR_EUNSUPPORTED; }
            if (nc == 2) {
                if (std::fabs(J[0] - J[4]) > lat->eps || std::fabs(J[0] - J[8]) > lat->eps) {
                    *msg = "tangent direction is not of Heisenberg form (SU2 core)"; return SR_EUNSUPPORTED;
                }
                (*out)[((size_t)r * 2 + 1) * npar + p] = J[8] / 4.0;
            } else {
                for (int c = 1; c < 4; ++c) (*out)[((size_t)r * 4 + c) * npar + p] = J[4 * (c - 1)] / 4.0;
            }
        }
        // every pair of every basis site must carry the value of its stored image
        for (size_t i = 0; i < lat->chi_sites.size(); ++i) {
            const int b = (int)(i / lat->Ntot);
            const SiteKey& j = lat->chi_sites[i];
            SiteKey d{{j.n[0], j.n[1], j.n[2]}, j.b};
            const auto J = pair_coupling(lat, b, d, Ms);
            const PairMap& pm = lat->chi_map[i];
            for (int c = 1; c < 4; ++c) {
                const int sc = nc == 2 ? 1 : pm.perm[c];
                const double img = (*out)[((size_t)pm.r * nc + sc) * npar + p] * 4.0;
                if (std::fabs(J[4 * (c - 1)] - img) > lat->eps) {
                    *msg = "tangent direction " + std::to_string(p) + " breaks a symmetry used to reduce the lattice";
                    return SR_ESYMMETRY;
                }
            }
        }
    }
    return SR_OK;
}

}  // namespace sr
