// Complex arithmetic and the chiral gamma matrices for code that runs on
// both the host and the device (the site arithmetic that host-only entry
// points share with their kernels).
#pragma once

struct zd {
    double re, im;
};
__host__ __device__ __forceinline__ zd zadd(zd a, zd b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ zd zsub(zd a, zd b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ zd zmulc(zd a, zd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__host__ __device__ __forceinline__ zd zconj(zd a) { return {a.re, -a.im}; }
__host__ __device__ __forceinline__ zd zscal(zd a, double s) { return {a.re * s, a.im * s}; }
__host__ __device__ __forceinline__ zd zdiv(zd a, zd b) {
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__host__ __device__ __forceinline__ double zabs(zd a) { return sqrt(a.re * a.re + a.im * a.im); }

// g_mu (4 x 4, row-major) in the chiral Euclidean basis of the library's
// hopping term: g_k = [[0, -i s_k], [i s_k, 0]] for mu = k - 1 = 0, 1, 2 (s_k
// the Pauli matrices), g_4 = [[0, 1], [1, 0]] for mu = 3
static inline void gamma_chiral(int mu, zd g[16]) {
    for (int i = 0; i < 16; ++i) g[i] = {0.0, 0.0};
    const zd P[3][4] = {{{0, 0}, {1, 0}, {1, 0}, {0, 0}},
                        {{0, 0}, {0, -1}, {0, 1}, {0, 0}},
                        {{1, 0}, {0, 0}, {0, 0}, {-1, 0}}};
    if (mu < 3) {
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const zd s = P[mu][2 * a + b];
                g[a * 4 + (b + 2)] = {s.im, -s.re};           // -i s
                g[(a + 2) * 4 + b] = {-s.im, s.re};           //  i s
            }
    } else {
        g[0 * 4 + 2] = g[1 * 4 + 3] = g[2 * 4 + 0] = g[3 * 4 + 1] = {1.0, 0.0};
    }
}

struct GammaTab {
    zd g[4][16];
};

static inline GammaTab make_gammas() {
    GammaTab T;
    for (int mu = 0; mu < 4; ++mu) gamma_chiral(mu, T.g[mu]);
    return T;
}

// link accessors: the library's packed FP64 links [4][9][N] (device) or the
// user layout [N][4][3][3]; entry e = 3 row + column
struct PackedLinks {
    const double *U;
    int N;
    __host__ __device__ __forceinline__ zd operator()(int site, int mu, int e) const {
        const size_t k = ((size_t)(mu * 9 + e) * N + site) * 2;
        return {U[k], U[k + 1]};
    }
};
struct UserLinks {
    const double *U;
    __host__ __device__ __forceinline__ zd operator()(int site, int mu, int e) const {
        const size_t k = (((size_t)site * 4 + mu) * 9 + e) * 2;
        return {U[k], U[k + 1]};
    }
};
