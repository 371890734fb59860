// Row-wise indexing of periodic grids [slice][z][y][x] (x fastest) for the
// one-level kernels.  A launch is a 2D grid: x comes from the thread index,
// the (slice, z, y) row from a grid-stride loop over blockIdx.y.  The integer
// divisions that split a row index happen once per row and are uniform across
// the block, so no point pays for a division; the periodic neighbours are a
// compare-and-select in x and constant offsets per row in y and z.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rows {

struct Row {
    int64_t slice_off;  // slice * pts
    int64_t off;        // first point of the row inside its slice: (z n + y) n
    int64_t yp, ym;     // offsets of rows y+1, y-1 (periodic) from the row (0 in 1D)
    int64_t zp, zm;     // offsets of planes z+1, z-1 (periodic) (0 below 3D)
};

// Row `row` of a batch whose slices hold pts = n^DIM points (n^(DIM-1) rows).
template <int DIM>
__device__ __forceinline__ Row row_of(int64_t row, int64_t n, int64_t pts) {
    Row r;
    r.yp = r.ym = r.zp = r.zm = 0;
    if (DIM == 1) {
        r.slice_off = row * pts;
        r.off = 0;
        return r;
    }
    const int64_t per_slice = pts / n;
    const int64_t s = row / per_slice;
    const int64_t q = row - s * per_slice;   // z n + y
    const int64_t z = DIM == 3 ? q / n : 0;
    const int64_t y = q - z * n;
    r.slice_off = s * pts;
    r.off = q * n;
    r.yp = (y + 1 == n ? -(n - 1) : 1) * n;
    r.ym = (y == 0 ? n - 1 : -1) * n;
    if (DIM == 3) {
        r.zp = (z + 1 == n ? -(n - 1) : 1) * n * n;
        r.zm = (z == 0 ? n - 1 : -1) * n * n;
    }
    return r;
}

// The 2*DIM periodic neighbours of point x of a row, as indices inside the
// slice, in the order +x, -x, +y, -y, +z, -z.
template <int DIM>
__device__ __forceinline__ void nbrs_of(const Row& r, int64_t x, int64_t n, int64_t* nb) {
    const int64_t p = r.off + x;
    nb[0] = p + (x + 1 == n ? -(n - 1) : 1);
    nb[1] = p + (x == 0 ? n - 1 : -1);
    if (DIM >= 2) {
        nb[2] = p + r.yp;
        nb[3] = p + r.ym;
    }
    if (DIM == 3) {
        nb[4] = p + r.zp;
        nb[5] = p + r.zm;
    }
}

// Launch shape for `total_rows` rows of n points: blocks of up to 256
// threads along x, and enough blocks along y for about four waves of a fully
// occupied GPU (each block then strides over the remaining rows).
inline void shape_for(int64_t n, int64_t total_rows, int sms, dim3* grid, dim3* block) {
    const int bx = n >= 256 ? 256 : (int)((n + 31) / 32 * 32);
    const int64_t gx = (n + bx - 1) / bx;
    int64_t gy = ((int64_t)sms * 2048 * 4 + bx * gx - 1) / (bx * gx);
    if (gy > total_rows) gy = total_rows;
    if (gy > 65535) gy = 65535;
    if (gy < 1) gy = 1;
    *grid = dim3((unsigned)gx, (unsigned)gy, 1);
    *block = dim3((unsigned)bx, 1, 1);
}

}  // namespace rows

namespace rows {

// Four consecutive points x0..x0+3 of a row (n % 4 == 0, x0 % 4 == 0) with
// their periodic neighbours: the quad itself, the points left of x0 and right
// of x0+3, and the quads of the rows y+-1 and planes z+-1.  128-bit loads for
// every quad, so a thread reads a point's 2*DIM neighbours with 1.75 load
// instructions per point instead of 2*DIM.
template <int DIM, typename T, typename V4>
struct Quad {
    V4 c, yp, ym, zp, zm;
    T l, r;
    // neighbour k (order +x, -x, +y, -y, +z, -z) of point j of the quad
    __device__ __forceinline__ T nb(int j, int k) const {
        switch (k) {
            case 0: return j == 3 ? r : comp(c, j + 1);
            case 1: return j == 0 ? l : comp(c, j - 1);
            case 2: return comp(yp, j);
            case 3: return comp(ym, j);
            case 4: return comp(zp, j);
            default: return comp(zm, j);
        }
    }
    __device__ __forceinline__ static T comp(const V4& v, int j) {
        return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
    }
};

// x-neighbour columns of the quad starting at x0 (periodic)
__device__ __forceinline__ void quad_edges(int64_t x0, int64_t n, int64_t* xl, int64_t* xr) {
    *xl = x0 == 0 ? n - 1 : x0 - 1;
    *xr = x0 + 4 == n ? 0 : x0 + 4;
}

template <int DIM, typename T, typename V4>
__device__ __forceinline__ Quad<DIM, T, V4> load_quad(const T* __restrict__ s, const Row& rw, int64_t x0,
                                                      int64_t xl, int64_t xr) {
    Quad<DIM, T, V4> q;
    const int64_t p = rw.off + x0;
    q.c = *(const V4*)(s + p);
    q.l = s[rw.off + xl];
    q.r = s[rw.off + xr];
    if (DIM >= 2) {
        q.yp = *(const V4*)(s + p + rw.yp);
        q.ym = *(const V4*)(s + p + rw.ym);
    }
    if (DIM == 3) {
        q.zp = *(const V4*)(s + p + rw.zp);
        q.zm = *(const V4*)(s + p + rw.zm);
    }
    return q;
}

}  // namespace rows
