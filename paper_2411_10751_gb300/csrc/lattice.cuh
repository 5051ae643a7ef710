// Velocity sets, quadrature weights and compile-time iteration helpers for
// the D2Q37 and D3Q39 lattices.
//
// D2Q37 (Sec. 4.1, Table 1): integer velocities on the shells
// |c|^2 in {0,1,2,4,5,8,9,10}.  The eight shell weights and s = c0^2 are the
// solution of the moment conditions of a degree-9 Gauss-Hermite rule with
// xi = c / c0: for even a, b with a + b <= 8,
//     sum_i w_i c_x^a c_y^b = s^((a+b)/2) (a-1)!! (b-1)!!.
// They are solved by lattice_gen.cpp when the library is built: for a fixed s
// the conditions of order <= 8 except (8,0) are linear in the weights (an
// 8 x 8 system); the (8,0) condition is then a scalar equation in s, solved by
// the secant method.  The result is compiled in as literal constants.
//
// D3Q39 (not in the paper): the standard degree-7 multi-speed lattice with
// closed-form weights 1/12, 1/12, 1/27, 2/135, 1/432, 1/1620 on the shells
// (0,0,0), (1,0,0), (1,1,1), (2,0,0), (2,2,0), (3,0,0) and c0^2 = 2/3.
//
// Both lattices are stored in "pair order": index 0 is the rest velocity and
// indices 2k+1, 2k+2 hold a velocity and its opposite.  The order has no
// physical meaning; it lets the collision share the even Hermite part between
// opposite velocities.
#pragma once

#include <cstdint>
#include <type_traits>

namespace hlbm {

// ---------------------------------------------------------------- unrolling
template <int... Is> struct iseq {};
template <int N, int... Is> struct make_iseq : make_iseq<N - 1, N - 1, Is...> {};
template <int... Is> struct make_iseq<0, Is...> { using type = iseq<Is...>; };

template <class F, int... Is>
__host__ __device__ __forceinline__ void static_for_impl(F&& f, iseq<Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
// Calls f(integral_constant<int, I>) for I = 0 .. N-1 (indices are constants).
template <int N, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, typename make_iseq<N>::type{});
}

// ------------------------------------------------------------ D2Q37 tables
namespace detail {

// Pair representatives of D2Q37 (each followed by its opposite).
__host__ __device__ constexpr int d2_pair(int p, int a) {
  constexpr int t[18][2] = {{1, 0},  {0, 1},  {1, 1},  {-1, 1}, {2, 0},  {0, 2},
                            {2, 1},  {1, 2},  {-1, 2}, {-2, 1}, {2, 2},  {-2, 2},
                            {3, 0},  {0, 3},  {3, 1},  {1, 3},  {-1, 3}, {-3, 1}};
  return t[p][a];
}

__host__ __device__ constexpr int d2_shell_of_norm(int n2) {
  return n2 == 0 ? 0 : n2 == 1 ? 1 : n2 == 2 ? 2 : n2 == 4 ? 3 : n2 == 5 ? 4 : n2 == 8 ? 5 : n2 == 9 ? 6 : 7;
}

// kD2W[8] (shell weights for |c|^2 = 0,1,2,4,5,8,9,10), kD2S (= c0^2) and kD2C0,
// written at build time by lattice_gen.cpp, which solves the moment
// conditions described at the top of this file.
#include "lattice_weights.inc"

__host__ __device__ constexpr double d2_shell_weight(int k) {
  constexpr double t[8] = {kD2W[0], kD2W[1], kD2W[2], kD2W[3], kD2W[4], kD2W[5], kD2W[6], kD2W[7]};
  return t[k];
}

}  // namespace detail

// ------------------------------------------------------------------ D2Q37
struct D2Q37 {
  static constexpr int D = 2;
  static constexpr int Q = 37;
  static constexpr int NPAIR = 18;
  static constexpr int REACH = 3;
  static constexpr int FEQ_ORDER = 4;   // Eq. 2.2 in full (degree-9 quadrature)
  static constexpr double cs2 = detail::kD2S;
  static constexpr double c0 = detail::kD2C0;

  __host__ __device__ static constexpr int c(int i, int a) {
    return a >= 2 ? 0
                  : (i == 0 ? 0
                            : (((i - 1) & 1) ? -detail::d2_pair((i - 1) >> 1, a)
                                             : detail::d2_pair((i - 1) >> 1, a)));
  }
  __host__ __device__ static constexpr int norm2(int i) { return c(i, 0) * c(i, 0) + c(i, 1) * c(i, 1); }
  __host__ __device__ static constexpr double w(int i) {
    return detail::d2_shell_weight(detail::d2_shell_of_norm(norm2(i)));
  }
};

// ------------------------------------------------------------------ D3Q39
namespace detail {
__host__ __device__ constexpr int d3_pair(int p, int a) {
  constexpr int t[19][3] = {
      {1, 0, 0}, {0, 1, 0}, {0, 0, 1},                                   // (1,0,0) x 6
      {1, 1, 1}, {-1, 1, 1}, {1, -1, 1}, {1, 1, -1},                     // (1,1,1) x 8
      {2, 0, 0}, {0, 2, 0}, {0, 0, 2},                                   // (2,0,0) x 6
      {2, 2, 0}, {2, -2, 0}, {2, 0, 2}, {2, 0, -2}, {0, 2, 2}, {0, 2, -2},  // (2,2,0) x 12
      {3, 0, 0}, {0, 3, 0}, {0, 0, 3}};                                  // (3,0,0) x 6
  return t[p][a];
}
__host__ __device__ constexpr double d3_weight_of_norm(int n2) {
  return n2 == 0 ? 1.0 / 12.0
       : n2 == 1 ? 1.0 / 12.0
       : n2 == 3 ? 1.0 / 27.0
       : n2 == 4 ? 2.0 / 135.0
       : n2 == 8 ? 1.0 / 432.0
                 : 1.0 / 1620.0;
}
}  // namespace detail

struct D3Q39 {
  static constexpr int D = 3;
  static constexpr int Q = 39;
  static constexpr int NPAIR = 19;
  static constexpr int REACH = 3;
  static constexpr int FEQ_ORDER = 3;   // degree-7 quadrature: third-order equilibrium
  static constexpr double cs2 = 2.0 / 3.0;
  static constexpr double c0 = 0.81649658092772603273242802490196;  // sqrt(2/3)

  __host__ __device__ static constexpr int c(int i, int a) {
    return i == 0 ? 0
                  : (((i - 1) & 1) ? -detail::d3_pair((i - 1) >> 1, a) : detail::d3_pair((i - 1) >> 1, a));
  }
  __host__ __device__ static constexpr int norm2(int i) {
    return c(i, 0) * c(i, 0) + c(i, 1) * c(i, 1) + c(i, 2) * c(i, 2);
  }
  __host__ __device__ static constexpr double w(int i) { return detail::d3_weight_of_norm(norm2(i)); }
};

}  // namespace hlbm
