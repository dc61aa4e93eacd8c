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

}  // namespace rlb
