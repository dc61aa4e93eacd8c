// rlb_consts.h -- lattice constants of the extended D3Q19 lattice, shared by
// host and device code.
#pragma once

namespace rlb {

// ---------------------------------------------------------------------------
// Lattice constants (Sec. II.A, Eqs. 42-46 and 59-60), nu = sqrt(13)
// ---------------------------------------------------------------------------
constexpr double kXi0 = 1.44115338424578420134928;      // c_t/c_0 = sqrt(27)/nu
constexpr double kXi0Sq = 27.0 / 13.0;
constexpr double kC0Ct = 0.693888666488710911760766;    // c_0/c_t
constexpr double kOmegaC = 2.50185116648837831287298;   // (c_0/c_t) nu = 13/sqrt(27)
constexpr double kFourOverXi0 = 2.77555466595484364704306;
constexpr double kPi2Over16 = 0.616850275068084913677156;  // 1 / (d_G / pi^2), d_G = 16
constexpr double kSMin = 1e-3;  // floor of 4 - ln(lambda) in the entropy density

// weights of f (Eqs. 43-45; independent of nu) and of h (Eqs. 59-60, c_a = 1)
constexpr double kW0 = -539.0 / 676.0, kW1 = 99.0 / 338.0, kW2 = 9.0 / 2704.0;
constexpr double kWh0 = 0.1, kWh1 = 6.0 / 35.0 - 1.0 / 42.0, kWh2 = 1.0 / 84.0 - 3.0 / 280.0;

// bulk coefficient alpha of Eq. 55 from zeta/s through Eq. 56 at the
// reference state T = 1, lambda = 1 (s = 4 n, P = n): alpha = 27 (zeta/s) / nu^6
inline double alpha_of_zeta(double zeta_over_s)
{
    return 27.0 * zeta_over_s / 2197.0;   // nu^6 = 13^3
}

// ---------------------------------------------------------------------------
// The two lattices, as compile-time traits: LAT = 0 the extended D3Q19
// configuration of Sec. II.A (diagonals 2 c_a, nu = sqrt(13)), LAT = 1 the
// basic D3Q19 lattice of Sec. II (diagonals c_a, nu = sqrt(19), c_a = 1).
// The equilibrium coefficients are the moment-matched ones (see
// rlb_device.cuh) with A = P / sigma2: 1/sigma2, the off-diagonal factor
// 4 sigma2 / m22 and the diagonal factor 4 sigma2 / (m4 - m22) of each
// lattice; the |u'|^2 factor -16/15 is the same on both.
// ---------------------------------------------------------------------------
template <int LAT>
struct Lat;

template <>
struct Lat<0> {
    static constexpr double nu2 = 13.0;
    static constexpr double nu6 = 2197.0;
    static constexpr double xi0 = kXi0;
    static constexpr double xi0sq = kXi0Sq;
    static constexpr double c0ct = kC0Ct;
    static constexpr double omegaC = kOmegaC;             // (c_0/c_t) nu
    static constexpr double four_over_xi0 = kFourOverXi0;
    static constexpr double inv_sigma2 = 13.0 / 9.0;
    static constexpr double a2f = 13.0;                   // 4 sigma2 / m22
    static constexpr double a3f = 52.0 / 15.0;            // 4 sigma2 / (m4 - m22)
    static constexpr double w0 = kW0, w1 = kW1, w2 = kW2;
    static constexpr double wh0 = kWh0, wh1 = kWh1, wh2 = kWh2;
    static constexpr int dmag = 2;                        // |c_ia| of a diagonal population
    // float forms for the FP32-storage kernel
    static constexpr float f_inv_sigma2 = 13.0f / 9.0f, f_a2f = 13.0f, f_a3f = 52.0f / 15.0f, f_nu2 = 13.0f;
};

template <>
struct Lat<1> {
    static constexpr double nu2 = 19.0;
    static constexpr double nu6 = 6859.0;
    static constexpr double xi0 = 1.19207912135853942587947655;  // c_t/c_0 = sqrt(27/19)
    static constexpr double xi0sq = 27.0 / 19.0;
    static constexpr double c0ct = 0.838870492807861077470742756; // sqrt(19/27)
    static constexpr double omegaC = 3.65655170486762984189127561;  // (c_0/c_t) nu = 19/sqrt(27)
    static constexpr double four_over_xi0 = 3.35548197123144430988297103; // 4 sqrt(19/27)
    static constexpr double inv_sigma2 = 19.0 / 9.0;
    static constexpr double a2f = 19.0;
    static constexpr double a3f = 76.0 / 15.0;
    static constexpr double w0 = -44.0 / 361.0, w1 = 99.0 / 722.0, w2 = 9.0 / 361.0;
    static constexpr double wh0 = 1.0 / 3.0, wh1 = 1.0 / 18.0, wh2 = 1.0 / 36.0;
    static constexpr int dmag = 1;
    static constexpr float f_inv_sigma2 = 19.0f / 9.0f, f_a2f = 19.0f, f_a3f = 76.0f / 15.0f, f_nu2 = 19.0f;
};

// alpha of Eq. 55 from zeta/s (Eq. 56) for either lattice
inline double alpha_of_zeta(double zeta_over_s, int lat)
{
    return 27.0 * zeta_over_s / (lat == 1 ? Lat<1>::nu6 : Lat<0>::nu6);
}

}  // namespace rlb
