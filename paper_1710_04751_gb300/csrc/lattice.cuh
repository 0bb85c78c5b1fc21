// lattice.cuh -- D3Q15 / D3Q7 velocity sets and the orthogonal collision matrices of
// arXiv:1710.04751 as compile-time functions, so that unrolled loops over directions
// and moments fold to straight-line adds and subtracts.
//
// Direction order (Sec. 2.2): 0 rest; 1,2 = +-x; 3,4 = +-y; 5,6 = +-z; 7..14 the cube
// diagonals with e_x alternating fastest, then e_y, then e_z (e_z = +1 for 7..10).
// D3Q7 (Appendix C) is directions 0..6.
#pragma once

namespace lbm {

__host__ __device__ constexpr int ex(int a) {
    return a == 1 ? 1 : a == 2 ? -1 : a >= 7 ? (((a - 7) & 1) ? -1 : 1) : 0;
}
__host__ __device__ constexpr int ey(int a) {
    return a == 3 ? 1 : a == 4 ? -1 : a >= 7 ? ((((a - 7) >> 1) & 1) ? -1 : 1) : 0;
}
__host__ __device__ constexpr int ez(int a) {
    return a == 5 ? 1 : a == 6 ? -1 : a >= 7 ? (((a - 7) >> 2) ? -1 : 1) : 0;
}
// opposite direction: rest -> rest, 1<->2, 3<->4, 5<->6, diagonal a <-> 21 - a
__host__ __device__ constexpr int opp(int a) {
    return a == 0 ? 0 : a <= 6 ? ((a & 1) ? a + 1 : a - 1) : 21 - a;
}
// index of a D3Q15 direction from its components (runtime use: specular walls)
__host__ __device__ inline int dir_index(int dx, int dy, int dz) {
    if (dx != 0 && dy != 0 && dz != 0) return 7 + (dx < 0) + 2 * (dy < 0) + 4 * (dz < 0);
    if (dx != 0) return dx > 0 ? 1 : 2;
    if (dy != 0) return dy > 0 ? 3 : 4;
    return dz > 0 ? 5 : 6;
}

// D3Q15 collision matrix entry K_b(e_a) (Sec. 2.2, the Gram-Schmidt basis K_0..K_14).
__host__ __device__ constexpr int k15(int b, int a) {
    return b == 0 ? 1
         : b == 1 ? ex(a)
         : b == 2 ? ey(a)
         : b == 3 ? ez(a)
         : b == 4 ? ex(a) * ey(a)
         : b == 5 ? ex(a) * ez(a)
         : b == 6 ? ey(a) * ez(a)
         : b == 7 ? ex(a) * ex(a) - ey(a) * ey(a)
         : b == 8 ? ex(a) * ex(a) + ey(a) * ey(a) - 2 * ez(a) * ez(a)
         : b == 9 ? ex(a) * ex(a) + ey(a) * ey(a) + ez(a) * ez(a) - 2
         : b == 10 ? ex(a) * (5 * (ex(a) * ex(a) + ey(a) * ey(a) + ez(a) * ez(a)) - 13)
         : b == 11 ? ey(a) * (5 * (ex(a) * ex(a) + ey(a) * ey(a) + ez(a) * ez(a)) - 13)
         : b == 12 ? ez(a) * (5 * (ex(a) * ex(a) + ey(a) * ey(a) + ez(a) * ez(a)) - 13)
         : b == 13 ? ex(a) * ey(a) * ez(a)
         : 30 * (ex(a) * ex(a) * ey(a) * ey(a) + ex(a) * ex(a) * ez(a) * ez(a) +
                 ey(a) * ey(a) * ez(a) * ez(a)) -
               40 * (ex(a) * ex(a) + ey(a) * ey(a) + ez(a) * ez(a)) + 32;
}

// D3Q7 collision matrix entry (Appendix C, K_0..K_6).
__host__ __device__ constexpr int k7(int b, int a) {
    return b == 0 ? 1
         : b == 1 ? ex(a)
         : b == 2 ? ey(a)
         : b == 3 ? ez(a)
         : b == 4 ? ex(a) * ex(a) - ey(a) * ey(a)
         : b == 5 ? ex(a) * ex(a) + ey(a) * ey(a) - 2 * ez(a) * ez(a)
         : 7 * (ex(a) * ex(a) + ey(a) * ey(a) + ez(a) * ez(a)) - 6;
}

// The raw-moment monomials e_x^m e_y^n e_z^p the cascades need, by moment id.
enum Mom { M0, MX, MY, MZ, MXY, MXZ, MYZ, MXX, MYY, MZZ, MXYY, MXXY, MXXZ, MXYZ, MXXYY };
__host__ __device__ constexpr int mono(int m, int a) {
    return m == M0 ? 1
         : m == MX ? ex(a)
         : m == MY ? ey(a)
         : m == MZ ? ez(a)
         : m == MXY ? ex(a) * ey(a)
         : m == MXZ ? ex(a) * ez(a)
         : m == MYZ ? ey(a) * ez(a)
         : m == MXX ? ex(a) * ex(a)
         : m == MYY ? ey(a) * ey(a)
         : m == MZZ ? ez(a) * ez(a)
         : m == MXYY ? ex(a) * ey(a) * ey(a)
         : m == MXXY ? ex(a) * ex(a) * ey(a)
         : m == MXXZ ? ex(a) * ex(a) * ez(a)
         : m == MXYZ ? ex(a) * ey(a) * ez(a)
         : ex(a) * ex(a) * ey(a) * ey(a);
}

// Squared norms of K_0..K_14 (D3Q15) and K_0..K_6 (D3Q7).
__host__ __device__ constexpr int norm15(int b) {
    return b == 0 ? 15 : b <= 3 ? 10 : b <= 6 ? 8 : b == 7 ? 4 : b == 8 ? 12 : b == 9 ? 18
         : b <= 12 ? 160 : b == 13 ? 8 : 1440;
}

}  // namespace lbm
