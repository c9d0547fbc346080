// flb_layout.cuh -- storage of one lattice in HBM.
//
// Nine SoA planes per buffer. Each plane has a one-node ghost frame so that the
// pull g_i(x) = f*_i(x - v_i) of every interior node is a plain shifted read,
// with no periodic wrap in the hot loop:
//
//   row yy = y + 1 for y in [-1, Ly]          (Ly + 2 rows)
//   col  c = x + kXO for x in [-1, Lx]        (interior rows start 128-byte aligned)
//   element (i, x, y) at  i * plane + (y + 1) * pitch + x + kXO
//
// A ghost cell holds a copy of the interior cell it wraps to. The step kernels
// keep the ghosts current themselves: a node whose streamed value leaves the
// interior (x + v_ix or y + v_iy outside the lattice) also writes it to the
// ghost cell its periodic image will pull from.
#pragma once

#include <cstdint>

#include "flb_device.cuh"

namespace flb {

constexpr int kXO = 32;   // column of x = 0 (128 bytes in FP32)

struct Geometry {
    int Lx, Ly;
    long long pitch;   // elements per row, multiple of 32, >= Lx + kXO + 1
    long long plane;   // pitch * (Ly + 2)
};

inline Geometry make_geometry(int Lx, int Ly) {
    Geometry g;
    g.Lx = Lx;
    g.Ly = Ly;
    g.pitch = (long long)((Lx + kXO + 1 + 31) / 32 * 32);   // ghost columns, 128-byte rows
    g.plane = g.pitch * (Ly + 2);                           // ghost rows
    return g;
}

__host__ __device__ __forceinline__ long long at(const Geometry& g, int i, int x, int y) {
    return (long long)i * g.plane + (long long)(y + 1) * g.pitch + (x + kXO);
}

// The cell the pull of f_i at interior node (x, y) reads: x - v_i, a ghost cell
// at the edge of the lattice. Every writer keeps these cells current (the step
// kernels and the state scatter write the ghost copies; a slab's ghost rows
// are written by the halo exchange), so readers of the pre-collision state use
// this cell rather than its periodic image.
__host__ __device__ __forceinline__ long long pull_at(const Geometry& g, int i, int x, int y) {
    return at(g, i, x - cvx(i), y - cvy(i));
}

__host__ __device__ __forceinline__ int wrap(int a, int L) {
    return a < 0 ? a + L : (a >= L ? a - L : a);
}

// Store value f_i = f*_i(x, y) (x, y interior) and, if the stream carries it
// out of the lattice, its ghost copy at the cell its periodic image pulls.
template <class T>
__host__ __device__ __forceinline__ void store_pop(T* dst, const Geometry& g, int i, int x, int y, T v) {
    dst[at(g, i, x, y)] = v;
    const int xd = x + cvx(i), yd = y + cvy(i);
    if (xd < 0 || xd >= g.Lx || yd < 0 || yd >= g.Ly) {
        const int xw = wrap(xd, g.Lx), yw = wrap(yd, g.Ly);
        dst[at(g, i, xw - cvx(i), yw - cvy(i))] = v;
    }
}

// Store the populations v[i] of interior node (x, y) at p[i plane] (p: the
// node's cell in plane 0) with the ghost copies of store_pop: population i
// that leaves through the left (right) edge is also pulled by its periodic
// image from column x + Lx (x - Lx), one that leaves through the bottom (top)
// edge from row y + Ly (y - Ly), both at a corner. The edge tests are per
// thread and the copies predicated, so nodes away from the edge pay only the
// tests.
template <class T>
__host__ __device__ __forceinline__ void store_node_ghosts(T* p, const Geometry& g, int x, int y, const T v[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) p[i * g.plane] = v[i];
    const bool eL = x == 0, eR = x == g.Lx - 1, eB = y == 0, eT = y == g.Ly - 1;
    if (!(eL || eR || eB || eT)) return;
    const long long sx = g.Lx, sy = (long long)g.Ly * g.pitch;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const bool lx = cvx(i) < 0 ? eL : (cvx(i) > 0 ? eR : false);
        const bool ly = cvy(i) < 0 ? eB : (cvy(i) > 0 ? eT : false);
        if (lx || ly) {
            long long o = i * g.plane;
            if (lx) o += cvx(i) < 0 ? sx : -sx;
            if (ly) o += cvy(i) < 0 ? sy : -sy;
            p[o] = v[i];
        }
    }
}

template <class T>
__host__ __device__ __forceinline__ void store_node(T* dst, const Geometry& g, int x, int y, const T f[9]) {
    store_node_ghosts(dst + at(g, 0, x, y), g, x, y, f);
}

}  // namespace flb
