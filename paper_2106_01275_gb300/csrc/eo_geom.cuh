// Half-lattice geometry of even-odd preconditioning, for code that runs on
// both the host and the device.  Half-lattice fields hold the sites of one
// parity in storage order; with D_0 even, the sites i and i ^ 1 have opposite
// parities, so site i is entry i >> 1 of its parity's half field.
#pragma once

#include <stdint.h>

// Division by a lattice extent without a hardware divide (Granlund and
// Montgomery, "Division by invariant integers using multiplication", PLDI
// 1994): with l = ceil(log2 d), p = 31 + l and m = ceil(2^p / d) < 2^32,
// floor(n / d) = floor(n m / 2^p) for every 0 <= n < 2^31.
struct EoDiv {
    uint32_t m, p;
};

static inline EoDiv make_eo_div(uint32_t d) {
    if (d == 0) d = 1;
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    EoDiv f;
    f.p = 31 + l;
    f.m = (uint32_t)(((1ull << f.p) + d - 1) / d);
    return f;
}

__host__ __device__ __forceinline__ int eo_div(const EoDiv &f, int n) {
    return (int)(((uint64_t)(uint32_t)n * f.m) >> f.p);
}

struct EoGeom {
    int D[4];
    int stride[4];
    int N, Nh;
    EoDiv half0, d1, d2;      // D_0 / 2, D_1, D_2
};

static inline EoGeom make_eo_geom(const int dims[4]) {
    EoGeom g;
    int s = 1;
    for (int mu = 0; mu < 4; ++mu) { g.D[mu] = dims[mu]; g.stride[mu] = s; s *= dims[mu]; }
    g.N = s;
    g.Nh = s / 2;
    g.half0 = make_eo_div((uint32_t)(dims[0] / 2));
    g.d1 = make_eo_div((uint32_t)dims[1]);
    g.d2 = make_eo_div((uint32_t)dims[2]);
    return g;
}

// storage index and coordinates of entry h of the half field of parity par
__host__ __device__ __forceinline__ int eo_full_site(const EoGeom &g, int par, int h, int x[4]) {
    const int half0 = g.D[0] >> 1;
    const int q = eo_div(g.half0, h);
    const int x0h = h - q * half0;
    const int q2 = eo_div(g.d1, q);
    x[1] = q - q2 * g.D[1];
    x[3] = eo_div(g.d2, q2);
    x[2] = q2 - x[3] * g.D[2];
    const int b = (par ^ (x[1] + x[2] + x[3])) & 1;
    x[0] = 2 * x0h + b;
    return 2 * h + b;
}

// storage index of x + s e_mu (s = +1 or -1), periodic
__host__ __device__ __forceinline__ int eo_neighbour(const EoGeom &g, int i, const int x[4], int mu, int s) {
    if (s > 0) return (x[mu] == g.D[mu] - 1) ? i - (g.D[mu] - 1) * g.stride[mu] : i + g.stride[mu];
    return (x[mu] == 0) ? i + (g.D[mu] - 1) * g.stride[mu] : i - g.stride[mu];
}

