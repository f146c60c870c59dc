// Host-side lattice truncation and symmetry analysis of the flow library (internal header).
//
// Implements Sec. 4.1 of arXiv:2109.13317: sites within bond distance L of a reference
// site, the lattice symmetries T (mapping any site to the reference site) and the point
// group U of the reference site lifted by a global permutation of the spin components,
// the irreducible site set N_s, and the tabulated lattice sums sum_j Gamma_{i1 j} Gamma_{j i2}.
#pragma once

#include <array>
#include <string>
#include <unordered_map>
#include <vector>

#include "sr.h"

namespace sr {

struct SiteKey {
    int n[3];
    int b;
    bool operator==(const SiteKey& o) const { return n[0] == o.n[0] && n[1] == o.n[1] && n[2] == o.n[2] && b == o.b; }
};

struct SiteKeyHash {
    size_t operator()(const SiteKey& k) const {
        size_t h = (size_t)(k.n[0] * 73856093) ^ (size_t)(k.n[1] * 19349663) ^ (size_t)(k.n[2] * 83492791) ^ (size_t)(k.b * 2654435761u);
        return h;
    }
};

// A symmetry acting on sites by integer arithmetic: (n, b) -> (M n + m[b], pb[b]), with the
// spin components mapped by the signed permutation (sp, sg) (sp[0] = 0, sg[0] = 1):
// J^{sp(mu) sp(nu)}_{g(i) g(j)} = sg(mu) sg(nu) J^{mu nu}_{i j}.  The SU2 and XYZ cores use
// unsigned permutations (sg = 1); the TRI core uses the proper rotations among the signed
// permutations, under which the flow of all 16 basis functions is covariant.
struct Sym {
    int M[3][3];
    std::vector<std::array<int, 3>> m;
    std::vector<int> pb;
    std::array<int, 4> sp;
    std::array<int, 4> sg{{1, 1, 1, 1}};
    SiteKey apply(const SiteKey& s) const;
};

using Perm = std::array<int, 4>;

// TRI core: component c = mu * 4 + nu of a pair read as stored component (m[c] & 15) of the
// pair's irreducible site, negated when bit 4 of m[c] is set.
using Map16 = std::array<int, 16>;

struct RpaEntry16 {
    int rA, rB;
    Map16 mA, mB;
};

struct PairMap16 {
    int r;      // irreducible site, -1 beyond range
    Map16 m;
};

struct RpaEntry {
    int rA, rB;
    Perm pA, pB;
};

struct PairMap {
    int r;      // irreducible site, -1 beyond range
    Perm perm;  // component c of the pair is stored component perm[c] of site r
};

}  // namespace sr

struct sr_lattice {
    double prim[3][3];
    int nb = 0;
    std::vector<double> basis;  // nb x 3
    std::vector<sr_bond> bonds;
    std::vector<sr_coupling> couplings;
    int L = 0;
    sr_backend backend = SR_SU2;
    int nc = 2;
    double eps = 1e-5;

    std::vector<sr::Sym> G0;  // point group of the reference site (basis 0, cell 0)
    std::vector<sr::Sym> T;   // T[b] maps (cell 0, basis b) onto the reference site

    std::vector<sr::SiteKey> sites;  // N_tot sites within range of the reference site, BFS order
    std::unordered_map<sr::SiteKey, int, sr::SiteKeyHash> site_index;
    std::vector<int> site_r;         // irreducible site of each site
    std::vector<sr::Perm> site_perm;  // component map of the pair (ref, site)

    int Ns = 0;
    std::vector<int> rep;             // site index of the representative of each irreducible site
    std::vector<int> mult;            // number of sites mapped to each irreducible site
    std::vector<int> swap_r;          // irreducible site of the exchanged pair (rep, ref)
    std::vector<sr::Perm> swap_perm;
    std::vector<sr::Perm> onsite_perm;  // component map of the pair (rep, rep) onto site 0
    std::vector<double> init_gamma;     // Ns x nc, J^{cc}/4 (TRI: J^{mu nu}/4) of the pair (ref, rep)

    // TRI core (nc = 16): signed component maps with the mu <-> nu transposition of the site
    // exchange folded into swap_map16
    std::vector<sr::Map16> site_map16;   // per site: (ref, site) onto its irreducible site
    std::vector<sr::Map16> swap_map16;   // per irreducible site r: component c of (ref, rep_r) at
                                         // exchanged frequencies reads transposed (rep_r, ref)
    std::vector<sr::Map16> onsite_map16; // per irreducible site: (rep, rep) onto site 0
    std::vector<sr::RpaEntry16> rpa16;   // lattice-sum entries, as rpa
    std::vector<sr::PairMap16> chi_map16;

    std::vector<int> rpa_off;          // Ns + 1
    std::vector<sr::RpaEntry> rpa;     // P entries, grouped by output site

    // correlation measurement: per basis b, sites within range of (0, b)
    int Ntot = 0;
    std::vector<sr::SiteKey> chi_sites;  // nb x Ntot
    std::vector<sr::PairMap> chi_map;    // nb x Ntot
    std::vector<double> chi_dr;          // nb x Ntot x 3: r_b - r_j
    std::vector<int> chi_onsite;         // nb x Ntot

    sr::PairMap map_pair(const sr::SiteKey& i1, const sr::SiteKey& i2) const;
    sr::PairMap16 map_pair16(const sr::SiteKey& i1, const sr::SiteKey& i2) const;
    void position(const sr::SiteKey& s, double out[3]) const;
};

namespace sr {
// Builds every table; returns SR_OK or an error with a message in *msg.
sr_status build_lattice(const sr_lattice_desc* d, sr_lattice* lat, std::string* msg);

// Derivative of the initial vertex J^{cc}/4 of every irreducible site along npar coupling
// directions dM (npar x n_couplings x 9, row-major 3x3 per coupling, in the order the
// couplings were given): out[(r * nc + c) * npar + p].  Fails with SR_ESYMMETRY if a
// direction is not invariant under the symmetries used for the site reduction.
sr_status tangent_init(const sr_lattice* lat, int npar, const double* dM, std::vector<double>* out, std::string* msg);
}  // namespace sr
