// Build-time generator of the D2Q37 quadrature weights (Sec. 4.1, Table 1).
//
// Solves, for the eight shell weights W_k (|c|^2 = 0,1,2,4,5,8,9,10) and
// s = c0^2, the moment conditions of a degree-9 Gauss-Hermite rule
//     sum_i w_i c_x^a c_y^b = s^((a+b)/2) (a-1)!! (b-1)!!,  a, b even, a + b <= 8.
// For fixed s the conditions (0,0),(2,0),(4,0),(2,2),(6,0),(4,2),(6,2),(4,4)
// are linear in W (solved by Gaussian elimination with partial pivoting); the
// remaining (8,0) condition is a scalar equation in s, solved by the secant
// method in long double.  Writes lattice_weights.inc (C++ literals) to the
// path given as argv[1].
#include <cmath>
#include <cstdio>

static const int kPairs[18][2] = {{1, 0},  {0, 1},  {1, 1},  {-1, 1}, {2, 0},  {0, 2},
                                  {2, 1},  {1, 2},  {-1, 2}, {-2, 1}, {2, 2},  {-2, 2},
                                  {3, 0},  {0, 3},  {3, 1},  {1, 3},  {-1, 3}, {-3, 1}};
// the last condition, (8,0), is the scalar residual in s; the first eight
// form a well-conditioned linear system for the weights
static const int kExp[9][2] = {{0, 0}, {2, 0}, {4, 0}, {2, 2}, {6, 0}, {4, 2}, {6, 2}, {4, 4}, {8, 0}};

static int shell(int n2) {
  return n2 == 0 ? 0 : n2 == 1 ? 1 : n2 == 2 ? 2 : n2 == 4 ? 3 : n2 == 5 ? 4 : n2 == 8 ? 5 : n2 == 9 ? 6 : 7;
}
static long double dfact(int n) {
  long double r = 1;
  for (int k = n - 1; k > 0; k -= 2) r *= k;
  return r;
}
static long double ipow(long double x, int n) {
  long double r = 1;
  for (int k = 0; k < n; ++k) r *= x;
  return r;
}

static long double M[9][8];

static void moments() {
  for (int j = 0; j < 9; ++j)
    for (int k = 0; k < 8; ++k) M[j][k] = 0;
  M[0][0] = 1;  // rest velocity contributes only to the zeroth moment
  for (int p = 0; p < 18; ++p)
    for (int sg = -1; sg <= 1; sg += 2) {
      int cx = sg * kPairs[p][0], cy = sg * kPairs[p][1];
      int k = shell(cx * cx + cy * cy);
      for (int j = 0; j < 9; ++j) M[j][k] += ipow(cx, kExp[j][0]) * ipow(cy, kExp[j][1]);
    }
}

static long double residual(long double s, long double W[8]) {
  long double A[8][9];
  for (int j = 0; j < 8; ++j) {
    for (int k = 0; k < 8; ++k) A[j][k] = M[j][k];
    A[j][8] = ipow(s, (kExp[j][0] + kExp[j][1]) / 2) * dfact(kExp[j][0]) * dfact(kExp[j][1]);
  }
  for (int c = 0; c < 8; ++c) {
    int piv = c;
    for (int r = c + 1; r < 8; ++r)
      if (fabsl(A[r][c]) > fabsl(A[piv][c])) piv = r;
    for (int k = 0; k < 9; ++k) {
      long double t = A[c][k];
      A[c][k] = A[piv][k];
      A[piv][k] = t;
    }
    for (int r = 0; r < 8; ++r) {
      if (r == c) continue;
      long double f = A[r][c] / A[c][c];
      for (int k = c; k < 9; ++k) A[r][k] -= f * A[c][k];
    }
  }
  for (int k = 0; k < 8; ++k) W[k] = A[k][8] / A[k][k];
  long double lhs = 0;
  for (int k = 0; k < 8; ++k) lhs += M[8][k] * W[k];
  return lhs - ipow(s, 4) * dfact(8);
}

int main(int argc, char** argv) {
  if (argc < 2) {
    std::fprintf(stderr, "usage: lattice_gen OUT.inc\n");
    return 2;
  }
  moments();
  long double W[8];
  long double s0 = 0.69L, s1 = 0.71L;
  long double r0 = residual(s0, W), r1 = residual(s1, W);
  for (int it = 0; it < 100 && r1 != r0; ++it) {
    long double s2 = s1 - r1 * (s1 - s0) / (r1 - r0);
    s0 = s1;
    r0 = r1;
    s1 = s2;
    r1 = residual(s1, W);
    if (fabsl(s1 - s0) < 1e-19L) break;
  }
  residual(s1, W);
  long double sum = W[0] + 4 * W[1] + 4 * W[2] + 4 * W[3] + 8 * W[4] + 4 * W[5] + 4 * W[6] + 8 * W[7];
  if (!(fabsl(sum - 1.0L) < 1e-15L) || !(s1 > 0.6L && s1 < 0.8L)) {
    std::fprintf(stderr, "lattice_gen: solve failed (sum %Lg, s %Lg)\n", sum, s1);
    return 1;
  }
  FILE* f = std::fopen(argv[1], "w");
  if (!f) return 1;
  std::fprintf(f, "// generated by lattice_gen.cpp: D2Q37 shell weights and c0^2\n");
  std::fprintf(f, "constexpr double kD2W[8] = {");
  for (int k = 0; k < 8; ++k) std::fprintf(f, "%.21Le%s", W[k], k < 7 ? ", " : "};\n");
  std::fprintf(f, "constexpr double kD2S = %.21Le;\n", s1);
  std::fprintf(f, "constexpr double kD2C0 = %.21Le;\n", sqrtl(s1));
  std::fclose(f);
  return 0;
}
