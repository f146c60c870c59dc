// Projected spin coefficients of the TRI core (internal header, host and device).
//
// All 16 basis functions Gamma^{mu nu} of Eq. (frg:parametrization) of arXiv:2109.13317 are
// stored as real numbers g^{mu nu} with Gamma^{mu nu} = i^{iota(mu, nu)} g^{mu nu}, iota = 1
// when exactly one of mu, nu is 0 (the imaginary class of Eq. frg:parametrizationBasis2p).
// The spin sums of Eq. (frg:flowexplicit:2particle) reduce to products of Pauli matrices,
// sigma^a sigma^b = i^{pexp(a, b)} sigma^{a xor b} (labels 0 = identity, 1 = x, 2 = y,
// 3 = z); every coefficient below is the resulting power of i, which for states of the right
// classes is even, i.e. a sign.  Derived by hand from the five terms:
//   s channel   out^{mu nu} = sum_{ab} A^{ab} B^{cd} i^{pexp(a,c) + pexp(b,d)},  c = a^mu, d = b^nu
//   u channel   out^{mu nu} = sum_{ab} A^{ab} B^{cd} i^{pexp(c,a) + pexp(b,d)},  c = a^mu, d = b^nu
//   t, lattice  out^{mu nu} = 2 sum_l A^{mu l} B^{l nu}
//   t, on-site  out^{mu nu} = sum_{lm} A^{mu l} C^{mn} i^{pexp(m,l) + pexp(m^l,n)},  n = m^l^nu
//   t, on-site  out^{mu nu} = sum_{lm} C^{kl} B^{m nu} i^{pexp(l,m) + pexp(l^m,k)},  k = mu^l^m
//   chi (exchange part) sum_l 2 i^{pexp(mu,l) + pexp(mu^l,nu)} E^{kl},  k = mu^nu^l
// times i^{iota(inputs) - iota(output)} for the real storage.
#pragma once

namespace sr {
namespace tri {

// exponent of i in sigma^a sigma^b = i^e sigma^{a ^ b}: xy = iz, yz = ix, zx = iy
__host__ __device__ constexpr int pexp(int a, int b) {
    return (a == 0 || b == 0 || a == b) ? 0 : ((a % 3) + 1 == b ? 1 : 3);
}
__host__ __device__ constexpr int iota(int a, int b) { return (a == 0) != (b == 0) ? 1 : 0; }
__host__ __device__ constexpr int iota(int c) { return iota(c >> 2, c & 3); }
// +1 / -1 for an even power of i (the odd powers do not occur)
__host__ __device__ constexpr int sgn_of(int e) { return ((e % 4) + 4) % 4 == 0 ? 1 : -1; }
__host__ __device__ constexpr bool even(int e) { return ((e % 4) + 4) % 2 == 0; }

// s channel: coefficient of A^{ab} B^{(a^mu)(b^nu)} in out^{mu nu}
__host__ __device__ constexpr int coef_s(int mu, int nu, int a, int b) {
    return sgn_of(pexp(a, a ^ mu) + pexp(b, b ^ nu) + iota(a, b) + iota(a ^ mu, b ^ nu) - iota(mu, nu));
}
// u channel: coefficient of A^{ab} B^{(a^mu)(b^nu)} in out^{mu nu}
__host__ __device__ constexpr int coef_u(int mu, int nu, int a, int b) {
    return sgn_of(pexp(a ^ mu, a) + pexp(b, b ^ nu) + iota(a, b) + iota(a ^ mu, b ^ nu) - iota(mu, nu));
}
// t channel lattice sum: coefficient of A^{mu l} B^{l nu} (without the factor 2)
__host__ __device__ constexpr int coef_t(int mu, int nu, int l) {
    return sgn_of(iota(mu, l) + iota(l, nu) - iota(mu, nu));
}
// first on-site term: coefficient of A^{mu l} C^{m (m^l^nu)}
__host__ __device__ constexpr int coef_o2(int mu, int nu, int l, int m) {
    return sgn_of(pexp(m, l) + pexp(m ^ l, m ^ l ^ nu) + iota(mu, l) + iota(m, m ^ l ^ nu) - iota(mu, nu));
}
// second on-site term: coefficient of C^{(mu^l^m) l} B^{m nu}
__host__ __device__ constexpr int coef_o3(int mu, int nu, int l, int m) {
    return sgn_of(pexp(l, m) + pexp(l ^ m, mu ^ l ^ m) + iota(mu ^ l ^ m, l) + iota(m, nu) - iota(mu, nu));
}
// correlation, exchange part: coefficient of E^{(mu^nu^l) l} in chi^{mu nu} (without the factor 2)
__host__ __device__ constexpr int coef_x(int mu, int nu, int l) {
    return sgn_of(pexp(mu, l) + pexp(mu ^ l, nu) + iota(mu ^ nu ^ l, l) - iota(mu, nu));
}
// the exponents above are even for every index combination (checked at compile time)
__host__ __device__ constexpr bool all_even() {
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = 0; nu < 4; ++nu)
            for (int a = 0; a < 4; ++a) {
                if (!even(iota(mu, a) + iota(a, nu) - iota(mu, nu))) return false;
                if (!even(pexp(mu, a) + pexp(mu ^ a, nu) + iota(mu ^ nu ^ a, a) - iota(mu, nu))) return false;
                for (int b = 0; b < 4; ++b) {
                    if (!even(pexp(a, a ^ mu) + pexp(b, b ^ nu) + iota(a, b) + iota(a ^ mu, b ^ nu) - iota(mu, nu))) return false;
                    if (!even(pexp(a ^ mu, a) + pexp(b, b ^ nu) + iota(a, b) + iota(a ^ mu, b ^ nu) - iota(mu, nu))) return false;
                    if (!even(pexp(b, a) + pexp(b ^ a, b ^ a ^ nu) + iota(mu, a) + iota(b, b ^ a ^ nu) - iota(mu, nu))) return false;
                    if (!even(pexp(a, b) + pexp(a ^ b, mu ^ a ^ b) + iota(mu ^ a ^ b, a) + iota(b, nu) - iota(mu, nu))) return false;
                }
            }
    return true;
}
static_assert(all_even(), "TRI spin coefficients must be real");

}  // namespace tri
}  // namespace sr
