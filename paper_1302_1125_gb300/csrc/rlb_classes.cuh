// rlb_classes.cuh -- the population classes of the exact symmetry
// reductions, shared by the FP32-storage and FP64 step kernels.
//
// Planes per distribution: NP = 19, or fewer under an exact symmetry of the
// state, when populations that the symmetry maps onto each other stay equal:
// * NP = 7, 1-D (u_y = u_z = 0, fields uniform in y and z): populations with
//   the same weight and the same c_x; classes rest, +x, -x, the four y/z axis
//   populations, the four diagonals with c_x = +2, the four with c_x = -2 and
//   the four y-z diagonals;
// * NP = 14, 2-D (u_z = 0, fields uniform in z, i.e. nz = 1): mirror images
//   in z; classes rest, +x, -x, +y, -y, {+z, -z}, the four x-y diagonals and
//   the pairs (+x, +-z), (-x, +-z), (+y, +-z), (-y, +-z).
// Class k is stored in the plane of its first population rep(k) and counts
// mult(k) populations.
#pragma once

namespace rlb {

template <int NP>
__host__ __device__ constexpr int rep(int k)
{
    if constexpr (NP == 19) {
        return k;
    } else if constexpr (NP == 14) {
        constexpr int r[14] = {0, 1, 2, 3, 4, 5, 7, 8, 9, 10, 11, 13, 15, 17};
        return r[k];
    } else {
        constexpr int r[7] = {0, 1, 2, 3, 7, 9, 15};
        return r[k];
    }
}
template <int NP>
__host__ __device__ constexpr int mult(int k)
{
    if constexpr (NP == 19) return 1;
    else if constexpr (NP == 14) return (k == 5 || k >= 10) ? 2 : 1;
    else return k < 3 ? 1 : 4;
}
// the reductions keep sum c_y f (NP != 7) and sum c_z f (NP == 19) only
// where they can be non-zero
template <int NP>
__host__ __device__ constexpr bool has_vy() { return NP != 7; }
template <int NP>
__host__ __device__ constexpr bool has_vz() { return NP == 19; }

}  // namespace rlb
