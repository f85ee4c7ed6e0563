// RD3Q41 velocity set on the body-centred-cubic grid (Sec. 5, Table 1 of
// Kolluru, Atif & Ansumali, arXiv 2201.05280), laid out for the GPU kernels.
//
// Ordering: index 0 is the rest velocity; indices 2k+1 and 2k+2 (k = 0..19)
// hold a velocity and its negative, so that the even and odd parts of every
// Hermite target are formed once per pair. Velocities are stored doubled
// (integers), since the half-velocity shell has components +-1/2.
#pragma once

namespace rpk {

constexpr int kQ = 41;
constexpr int kPairs = 20;

// Sec. 5, Table 1 caption.
constexpr double kTheta0 = 0.2948964908710633;

struct Vel2 {
  int x, y, z;  // 2 * c
};

// One representative of each +-pair; the partner is its negative.
constexpr Vel2 kPairVel2[kPairs] = {
    // |c| = 1 along an axis
    {2, 0, 0}, {0, 2, 0}, {0, 0, 2},
    // |c| = 2 along an axis
    {4, 0, 0}, {0, 4, 0}, {0, 0, 4},
    // (+-1, +-1, 0) and permutations
    {2, 2, 0}, {2, -2, 0}, {2, 0, 2}, {2, 0, -2}, {0, 2, 2}, {0, 2, -2},
    // (+-1, +-1, +-1)
    {2, 2, 2}, {2, 2, -2}, {2, -2, 2}, {2, -2, -2},
    // (+-1/2, +-1/2, +-1/2): these hop between the two sublattices
    {1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {1, -1, -1},
};

// Table 1 weights as functions of theta0, one per shell.
__host__ __device__ constexpr double weight_rest(double t) {
  return (52.0 - 323.0 * t + 921.0 * t * t - 1036.0 * t * t * t) / 52.0;
}
__host__ __device__ constexpr double weight_axis1(double t) { return t * (12.0 - 38.0 * t + 63.0 * t * t) / 39.0; }
__host__ __device__ constexpr double weight_axis2(double t) { return t * (3.0 - 29.0 * t + 84.0 * t * t) / 312.0; }
__host__ __device__ constexpr double weight_face(double t) { return t * (45.0 * t - 6.0 - 77.0 * t * t) / 26.0; }
__host__ __device__ constexpr double weight_corner(double t) { return t * (20.0 - 163.0 * t + 378.0 * t * t) / 312.0; }
__host__ __device__ constexpr double weight_half(double t) { return 8.0 * t * (4.0 - 17.0 * t + 21.0 * t * t) / 39.0; }

// Weight of pair k (both members share it).
__host__ __device__ constexpr double pair_weight(int k) {
  return k < 3    ? weight_axis1(kTheta0)
         : k < 6  ? weight_axis2(kTheta0)
         : k < 12 ? weight_face(kTheta0)
         : k < 16 ? weight_corner(kTheta0)
                  : weight_half(kTheta0);
}
constexpr double kWeightRest = weight_rest(kTheta0);

__host__ __device__ constexpr bool pair_is_half(int k) { return k >= 16; }

// Velocity of population q in the kernel ordering, doubled.
__host__ __device__ constexpr Vel2 vel2(int q) {
  return q == 0 ? Vel2{0, 0, 0}
         : (q & 1) ? kPairVel2[(q - 1) / 2]
                   : Vel2{-kPairVel2[(q - 1) / 2].x, -kPairVel2[(q - 1) / 2].y,
                          -kPairVel2[(q - 1) / 2].z};
}
__host__ __device__ constexpr double weight(int q) { return q == 0 ? kWeightRest : pair_weight((q - 1) / 2); }

}  // namespace rpk
