// Test helper: runs the lattice layout's index arithmetic (flb_layout.cuh, the
// code the kernels use) on the host. For a lattice of Lx x Ly it stores a
// distinct value for every (plane, node) with store_node, then pulls every
// node's nine populations the way the step kernels do and counts mismatches
// against the value its periodic origin stored, and out-of-range indices.
#include <cstdio>
#include <vector>

#include "../../paper_1204_6734_gb300/csrc/flb_layout.cuh"

using namespace flb;

extern "C" long long layout_check(int Lx, int Ly, long long* pitch_out, long long* plane_out) {
    const Geometry g = make_geometry(Lx, Ly);
    if (pitch_out) *pitch_out = g.pitch;
    if (plane_out) *plane_out = g.plane;
    const long long total = 9 * g.plane;
    std::vector<double> buf(total, -1.0);
    long long bad = 0;
    auto value = [&](int i, int x, int y) { return 1.0 + i + 10.0 * x + 1e5 * y; };
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            double f[9];
            for (int i = 0; i < 9; ++i) f[i] = value(i, x, y);
            // bounds of every index store_node may touch
            for (int i = 0; i < 9; ++i) {
                const long long k = at(g, i, x, y);
                if (k < 0 || k >= total) ++bad;
                const int xd = x + cvx(i), yd = y + cvy(i);
                const long long kg = at(g, i, wrap(xd, Lx) - cvx(i), wrap(yd, Ly) - cvy(i));
                if (kg < 0 || kg >= total) ++bad;
            }
            if (bad) return -bad;
            store_node(buf.data(), g, x, y, f);
        }
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x)
            for (int i = 0; i < 9; ++i) {
                const long long k = at(g, i, x - cvx(i), y - cvy(i));
                if (k < 0 || k >= total) return -1000000;
                const int ox = wrap(x - cvx(i), Lx), oy = wrap(y - cvy(i), Ly);
                if (buf[k] != value(i, ox, oy)) ++bad;
            }
    return bad;
}
