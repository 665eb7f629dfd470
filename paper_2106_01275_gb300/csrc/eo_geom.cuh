// Half-lattice geometry of even-odd preconditioning, for code that runs on
// both the host and the device.  Half-lattice fields hold the sites of one
// parity in storage order; with D_0 even, the sites i and i ^ 1 have opposite
// parities, so site i is entry i >> 1 of its parity's half field.
#pragma once

struct EoGeom {
    int D[4];
    int stride[4];
    int N, Nh;
};

static inline EoGeom make_eo_geom(const int dims[4]) {
    EoGeom g;
    int s = 1;
    for (int mu = 0; mu < 4; ++mu) { g.D[mu] = dims[mu]; g.stride[mu] = s; s *= dims[mu]; }
    g.N = s;
    g.Nh = s / 2;
    return g;
}

// storage index and coordinates of entry h of the half field of parity par
__host__ __device__ __forceinline__ int eo_full_site(const EoGeom &g, int par, int h, int x[4]) {
    const int half0 = g.D[0] >> 1;
    const int q = h / half0;
    const int x0h = h - q * half0;
    x[1] = q % g.D[1];
    const int q2 = q / g.D[1];
    x[2] = q2 % g.D[2];
    x[3] = q2 / g.D[2];
    const int b = (par ^ (x[1] + x[2] + x[3])) & 1;
    x[0] = 2 * x0h + b;
    return 2 * h + b;
}

// storage index of x + s e_mu (s = +1 or -1), periodic
__host__ __device__ __forceinline__ int eo_neighbour(const EoGeom &g, int i, const int x[4], int mu, int s) {
    if (s > 0) return (x[mu] == g.D[mu] - 1) ? i - (g.D[mu] - 1) * g.stride[mu] : i + g.stride[mu];
    return (x[mu] == 0) ? i + (g.D[mu] - 1) * g.stride[mu] : i - g.stride[mu];
}

