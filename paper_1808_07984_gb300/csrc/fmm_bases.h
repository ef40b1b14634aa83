// fmm_bases.h -- one-level bases given as coefficient tables, and the parameters of the
// operand-sum pass that forms their products' operands from a table at run time.
//
// A basis <g_m, g_k, g_n; R> splits A into a g_m x g_k grid of blocks, B into g_k x g_n and
// C into g_m x g_n, and forms R products M_r = (sum_a U[a][r] A_a)(sum_b V[b][r] B_b), each
// added into C block c with coefficient W[c][r]; blocks are numbered row-major in their grid
// (a = i*g_k + l, b = l*g_n + j, c = i*g_n + j).  Section 6 names bases other than Strassen's
// <2,2,2; 7> as what the same primitive can carry next.
#pragma once
#include <cstdint>
#include "fmm_kernels.cuh"

namespace fmm {

// fmm_options.basis values beyond kBasisStrassen (0) and kBasisWinograd (1)
constexpr int kBasis323 = 2;
// <2,3,2; 11>: A split into 2 x 3 blocks, B into 3 x 2, C into 2 x 2; eleven products where
// the classical scheme needs twelve (the least possible for this shape).  Products 0..6 are
// Strassen's Eq. 3 on the first two block columns of A and block rows of B; products 7..10
// add the outer product A(:, 2) B(2, :) block by block: M_{7 + 2i + j} = A(i,2) B(2,j) into
// C(i,j).  Built from the Strassen tables in make_products (no separate table).
constexpr int kBasis232 = 3;

constexpr int kMaxTableBlocks = 9;  // source blocks of one operand in a table pass
constexpr int kMaxTableRank = 32;   // products of one table pass

// <3,2,3; 15>: fifteen products where the classical scheme needs eighteen (the least
// possible for <3,2,3>, Hopcroft and Kerr).  Found for this library by a random walk over
// rank-reducing rewrites of the classical scheme modulo 2, followed by a choice of signs;
// it is exact because it satisfies the Brent equations (checked by the tests against the
// same equations), not by that search.  Every product feeds at most three C blocks.
// Rows: blocks; columns: products 0..14.
constexpr int8_t kB323U[6][15] = {
    {-1, 1, 1, -1, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0},    // A(0,0)
    {0, 1, 1, 0, -1, 0, 0, 0, 0, 1, 1, 0, 0, 0, 1},     // A(0,1)
    {0, 0, 0, 1, -1, 1, 0, 0, 0, 0, 0, -1, -1, 1, 0},   // A(1,0)
    {0, 0, 0, 0, 0, 1, 0, 0, -1, 0, -1, -1, -1, 0, 0},  // A(1,1)
    {1, -1, -1, 0, 0, 0, 0, -1, 0, 0, 0, 0, 1, 0, 0},   // A(2,0)
    {0, 0, -1, 0, 0, -1, 1, 0, 1, 0, 0, 0, 1, 0, 0},    // A(2,1)
};
constexpr int8_t kB323V[6][15] = {
    {1, 0, 0, 0, 0, -1, 0, -1, 1, 0, 0, 0, 1, 0, 0},     // B(0,0)
    {0, 0, 0, 1, 0, -1, 0, 0, 1, 0, 0, 0, 1, 1, 0},      // B(0,1)
    {-1, 1, 0, -1, -1, 0, 0, 0, 0, -1, 0, 0, 0, 0, -1},  // B(0,2)
    {-1, 1, 1, 0, 0, 0, -1, 0, -1, 0, 0, 0, 0, 0, 0},    // B(1,0)
    {0, 0, 0, 0, 1, 1, 0, 0, -1, 0, -1, 1, 0, -1, 0},    // B(1,1)
    {1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 1},     // B(1,2)
};
constexpr int8_t kB323W[9][15] = {
    {-1, 1, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 1},    // C(0,0)
    {0, 0, 0, -1, -1, 0, 0, 0, 0, -1, 0, 0, 0, 1, 0},  // C(0,1)
    {0, 0, 0, 0, 0, 0, 0, 0, 0, -1, 0, 0, 0, 0, 1},    // C(0,2)
    {0, 0, 0, 0, 0, -1, -1, 0, 1, 0, 0, 0, 0, -1, 0},  // C(1,0)
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1, 0, 1, 0},    // C(1,1)
    {0, 0, 0, 0, 1, 0, 0, 0, 0, 0, -1, -1, 0, 0, 1},   // C(1,2)
    {0, 0, 0, 0, 0, 0, -1, 1, 0, 0, 0, 0, 0, 0, 0},    // C(2,0)
    {0, 0, 0, 0, 0, -1, 0, -1, 0, 0, 0, -1, 1, 0, 0},  // C(2,1)
    {0, -1, 1, 0, 0, 0, -1, 0, 0, -1, 0, 0, 0, 0, 0},  // C(2,2)
};

// Parameters of the table-driven operand-sum pass over one operand: the stored source is a
// grid_r x grid_c grid of p.hr x p.hc blocks (zero outside the source), and product r's sum
// is sum_s coef[s][r] * X_s over stored blocks s = br * grid_c + bc.  Stored-block order
// already accounts for a source stored transposed.  Coefficients are -1, 0 or 1.
struct TableSumParams {
  SumParams p;
  int32_t grid_r, grid_c;
  int32_t nprod;
  int8_t coef[kMaxTableBlocks][kMaxTableRank];
};

}  // namespace fmm
