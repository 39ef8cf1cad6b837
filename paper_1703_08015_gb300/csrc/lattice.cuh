// lattice.cuh -- compile-time lattice tables and tile geometry for the
// device kernels.
//
// The links follow the order documented in include/lbm.h.  All loops over
// links go through static_for, so every c_i, w_i and opp(i) below is a
// compile-time constant in the generated code.
#pragma once

#include <cstdint>
#include <type_traits>

namespace lbm {

template <int Begin, int End, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
    if constexpr (Begin < End) {
        f(std::integral_constant<int, Begin>{});
        static_for<Begin + 1, End>(f);
    }
}

// D2Q9: rest, 4 axis links, 4 diagonals (weights 4/9, 1/9, 1/36).
struct D2Q9 {
    static constexpr int D = 2, Q = 9;
    static constexpr int cx_[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    static constexpr int cy_[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    static constexpr int cz_[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    static constexpr int opp_[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    // weight class of each link: 0 = rest, 1 = axis, 2 = diagonal
    static constexpr int cls_[9] = {0, 1, 1, 1, 1, 2, 2, 2, 2};
    static constexpr double wc_[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
};

// D3Q19: rest, 6 axis links, 12 edge diagonals in +- pairs
// (weights 1/3, 1/18, 1/36).
struct D3Q19 {
    static constexpr int D = 3, Q = 19;
    static constexpr int cx_[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    static constexpr int cy_[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    static constexpr int cz_[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    static constexpr int opp_[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
    static constexpr int cls_[19] = {0, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2};
    static constexpr double wc_[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
};

template <class L, int I>
struct Link {
    static constexpr int cx = L::cx_[I];
    static constexpr int cy = L::cy_[I];
    static constexpr int cz = L::cz_[I];
    static constexpr int opp = L::opp_[I];
    static constexpr int cls = L::cls_[I];
    static constexpr double w = L::wc_[L::cls_[I]];
};

__host__ __device__ constexpr int ipow(int a, int d) { return d == 0 ? 1 : a * ipow(a, d - 1); }
__host__ __device__ constexpr int ilog2(int a) { return a <= 1 ? 0 : 1 + ilog2(a / 2); }

// Geometry of one tile of A^D nodes, node index n = lx + A*ly + A*A*lz.
template <class L, int A>
struct Tile {
    static constexpr int D = L::D;
    static constexpr int NT = ipow(A, D);          // nodes per tile (n_tn)
    static constexpr int NN = (D == 3) ? 27 : 9;   // neighbour slots (3^d)
    static constexpr int CENTER = (D == 3) ? 13 : 4;
    static constexpr int W = (NT + 63) / 64;        // 64-bit mask words per tile
    static constexpr int LA = ilog2(A);
    static_assert((1 << LA) == A, "tile edge must be a power of two");
};

}  // namespace lbm
