// Test helper: exposes the CUDA toolkit's own Philox4x32-10 (curand_Philox4x32_10
// from curand_philox4x32_x.h) as a host function, so that the oracle's Philox can
// be checked against an implementation that is not ours. Compiled for the host
// only; the header's functions are called, not copied.
#define QUALIFIERS static __forceinline__ __host__ __device__
#include <curand_philox4x32_x.h>

extern "C" void ref_philox4x32_10(const unsigned* ctr, const unsigned* key, unsigned* out, int n) {
    for (int k = 0; k < n; ++k) {
        uint4 c = make_uint4(ctr[4 * k], ctr[4 * k + 1], ctr[4 * k + 2], ctr[4 * k + 3]);
        uint2 kk = make_uint2(key[2 * k], key[2 * k + 1]);
        uint4 r = curand_Philox4x32_10(c, kk);
        out[4 * k] = r.x; out[4 * k + 1] = r.y; out[4 * k + 2] = r.z; out[4 * k + 3] = r.w;
    }
}
