// t4grid.cuh - complex grids in global scratch stored in 4 x 4 tiles, for passes
// that a half-warp runs along rows and along columns in turn.
//
// Element (r, c) of a grid with ncols columns (a multiple of 4; rows allocated in
// groups of 4) sits in the 128-byte line of tile (r / 4, c / 4), in its 32-byte sector
// of rows 2 (r / 2) .. +1 and columns 2 (c / 2) .. +1. A warp's two half-warps reading
// or writing two adjacent rows over 16 columns (rows 2 w' and 2 w' + 1), or two
// adjacent columns over 16 rows, touch 4 or 5 lines per instruction and use every
// sector they load; a row-major grid gives the columns 16 lines and half-used sectors
// per instruction (bound by the L1 pipeline), the rows 2 lines.
// t4_index(r, c) = t4_row(r, ncols) + t4_col(c); adding 4 k to c adds 16 k, and rows
// congruent mod 4 share their in-tile offset t4_low.
#pragma once

namespace apic {

__device__ __forceinline__ int t4_low(int r) { return ((r & 2) << 2) + ((r & 1) << 1); }
__device__ __forceinline__ int t4_row(int r, int ncols) { return (r & ~3) * ncols + t4_low(r); }
__device__ __forceinline__ int t4_col(int c) { return ((c & ~3) << 2) + ((c & 2) << 1) + (c & 1); }
__device__ __forceinline__ int t4_index(int r, int c, int ncols) { return t4_row(r, ncols) + t4_col(c); }
__host__ __device__ inline int t4_rows(int rows) { return (rows + 3) & ~3; }

// Offset of column t + m of a row (lane t; m known after unrolling): the lane's four
// column offsets t4_col(t + q), q < 4, and a multiple of 16.
struct T4Lane {
    int c0, c1, c2, c3;
    __device__ explicit T4Lane(int t) : c0(t4_col(t)), c1(t4_col(t + 1)), c2(t4_col(t + 2)), c3(t4_col(t + 3)) {}
    __device__ __forceinline__ int at(int m) const {
        const int q = m & 3;
        return (q == 0 ? c0 : q == 1 ? c1 : q == 2 ? c2 : c3) + 4 * (m & ~3);
    }
};

}  // namespace apic
