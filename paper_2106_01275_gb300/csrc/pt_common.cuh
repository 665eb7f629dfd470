// Internal definitions shared by the CUDA translation units of libptrace.
//
// Internal field layout (structure of arrays; element (component c, site x)
// is reached through ld_cx / st_cx, so copies in different precisions convert
// component by component):
//   scalar field (dof 1):  real [N]
//   spinor field (dof 12), component a = 3 * spin + colour, complex (re, im):
//     FP64, BF16: [12 components][N sites]
//     FP32:       [6 pairs of components][N sites] of 16-byte chunks, so that a
//                 site's spinor is six 16-byte loads
//   links:
//     FP64, BF16: complex [4 mu][9 = 3 row x 3 col][N]
//     FP32:       [4 mu][5][N] 16-byte chunks holding entries (2k, 2k+1), the
//                 tenth entry is padding (zero)
// One right-hand side ("slot") of the batched solver owns one such field per
// Krylov vector; slot j starts at j * L reals, L = N (scalar) or 24 N (spinor).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/ptrace.h"

#define PT_MAX_P 32          // displacements (times nested levels) contracted in one call
#define PT_BS 128            // sites per CTA work item

// ------------------------------------------------------------------ errors
void pt_set_error(const char *fmt, ...);
int pt_cuda_fail(cudaError_t e, const char *what, const char *file, int line);
#define PT_CUDA(call)                                                           \
    do {                                                                        \
        cudaError_t _e = (call);                                                \
        if (_e != cudaSuccess) return pt_cuda_fail(_e, #call, __FILE__, __LINE__); \
    } while (0)
#define PT_CHECK_ARG(cond, ...)                                                 \
    do {                                                                        \
        if (!(cond)) { pt_set_error(__VA_ARGS__); return PT_ERR_ARG; }          \
    } while (0)

// ------------------------------------------------------------------ geometry
// Division by a lattice extent without a hardware divide (Granlund and
// Montgomery, "Division by invariant integers using multiplication", PLDI
// 1994): with l = ceil(log2 d), p = 31 + l and m = ceil(2^p / d) < 2^32,
// floor(n / d) = floor(n m / 2^p) for every 0 <= n < 2^31.
struct FastDiv {
    uint32_t d, m, p;
};

static inline FastDiv make_fastdiv(uint32_t d) {
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    FastDiv f;
    f.d = d;
    f.p = 31 + l;
    f.m = (uint32_t)(((1ull << f.p) + d - 1) / d);
    return f;
}

__device__ __forceinline__ int fdiv(const FastDiv &f, int n) {
    return (int)(((uint64_t)(uint32_t)n * f.m) >> f.p);
}

struct Geom {
    int D[4];
    int stride[4];
    int N;
    FastDiv fd[3];
};

static inline Geom make_geom(const int dims[4]) {
    Geom g;
    int s = 1;
    for (int mu = 0; mu < 4; ++mu) { g.D[mu] = dims[mu]; g.stride[mu] = s; s *= dims[mu]; }
    g.N = s;
    for (int mu = 0; mu < 3; ++mu) g.fd[mu] = make_fastdiv((uint32_t)dims[mu]);
    return g;
}

__device__ __forceinline__ void site_coords(const Geom &g, int idx, int x[4]) {
    int q0 = fdiv(g.fd[0], idx);
    x[0] = idx - q0 * g.D[0];
    int q1 = fdiv(g.fd[1], q0);
    x[1] = q0 - q1 * g.D[1];
    int q2 = fdiv(g.fd[2], q1);
    x[2] = q1 - q2 * g.D[2];
    x[3] = q2;
}

__device__ __forceinline__ int nb_fwd(const Geom &g, int idx, const int x[4], int mu) {
    return (x[mu] == g.D[mu] - 1) ? idx - (g.D[mu] - 1) * g.stride[mu] : idx + g.stride[mu];
}
__device__ __forceinline__ int nb_bwd(const Geom &g, int idx, const int x[4], int mu) {
    return (x[mu] == 0) ? idx + (g.D[mu] - 1) * g.stride[mu] : idx - g.stride[mu];
}
// idx of x + p e_mu (mod D), any integer p
__device__ __forceinline__ int shift_site(const Geom &g, int idx, const int x[4], int mu, int p) {
    int c = (x[mu] + p) % g.D[mu];
    if (c < 0) c += g.D[mu];
    return idx + (c - x[mu]) * g.stride[mu];
}

// ------------------------------------------------------------------ complex helpers
template <typename R> struct Cx { R re, im; };
template <typename R> __device__ __forceinline__ Cx<R> cmk(R a, R b) { return Cx<R>{a, b}; }
template <typename R> __device__ __forceinline__ Cx<R> cadd(Cx<R> a, Cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __device__ __forceinline__ Cx<R> csub(Cx<R> a, Cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> __device__ __forceinline__ Cx<R> cconjmul(Cx<R> a, Cx<R> b) {  // conj(a) b
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename R> __device__ __forceinline__ Cx<R> ctimes_i(Cx<R> a) { return {-a.im, a.re}; }
template <typename R> __device__ __forceinline__ Cx<R> cscale(Cx<R> a, R s) { return {a.re * s, a.im * s}; }

// ------------------------------------------------------------------ SplitMix64 noise
// Steele, Lea, Flood (OOPSLA 2014): output n of a generator at state S is
// mix64(S + n * GAMMA).  key(seed, set) = output set+1 from `seed`;
// h(x) = output x+1 from key.  Z2: 1 - 2 (h >> 63).  Z4: i^(h >> 62).
#define PT_GAMMA 0x9E3779B97F4A7C15ULL
__host__ __device__ __forceinline__ uint64_t pt_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t pt_set_key(uint64_t seed, int set) {
    return pt_mix64(seed + (uint64_t)(set + 1) * PT_GAMMA);
}
// noise value for counter c (site index, or dof * site + component when undiluted)
__device__ __forceinline__ Cx<double> pt_noise(uint64_t key, uint64_t c, int kind) {
    uint64_t h = pt_mix64(key + (c + 1ULL) * PT_GAMMA);
    if (kind == PT_NOISE_Z2) return Cx<double>{(h >> 63) ? -1.0 : 1.0, 0.0};
    switch ((int)(h >> 62)) {
        case 0: return Cx<double>{1.0, 0.0};
        case 1: return Cx<double>{0.0, 1.0};
        case 2: return Cx<double>{-1.0, 0.0};
        default: return Cx<double>{0.0, -1.0};
    }
}

// ------------------------------------------------------------------ storage types
// Element type of a real array in a given precision.
template <int PREC> struct StoreT;
template <> struct StoreT<PT_PREC_FP64> { typedef double T; };
template <> struct StoreT<PT_PREC_MIXED_FP32> { typedef float T; };
template <> struct StoreT<PT_PREC_MIXED_BF16> { typedef __nv_bfloat16 T; };

// arithmetic type for a storage type: FP64 stays FP64, FP32 and BF16 compute in FP32
template <typename S> struct ArithT { typedef float T; };
template <> struct ArithT<double> { typedef double T; };

__device__ __forceinline__ float ld_real(const float *p, size_t i) { return p[i]; }
__device__ __forceinline__ double ld_real(const double *p, size_t i) { return p[i]; }
__device__ __forceinline__ float ld_real(const __nv_bfloat16 *p, size_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ void st_real(float *p, size_t i, float v) { p[i] = v; }
__device__ __forceinline__ void st_real(double *p, size_t i, double v) { p[i] = v; }
__device__ __forceinline__ void st_real(__nv_bfloat16 *p, size_t i, float v) { p[i] = __float2bfloat16_rn(v); }

// complex element (component c, site idx) of a spinor field with N sites
template <typename S, typename R>
__device__ __forceinline__ Cx<R> ld_cx(const S *f, int N, int c, int idx);
template <>
__device__ __forceinline__ Cx<float> ld_cx<float, float>(const float *f, int N, int c, int idx) {
    // FP32: component pairs in 16-byte chunks [c / 2][idx], half c % 2
    float2 v = reinterpret_cast<const float2 *>(f)[((size_t)(c >> 1) * N + idx) * 2 + (c & 1)];
    return Cx<float>{v.x, v.y};
}
template <>
__device__ __forceinline__ Cx<double> ld_cx<double, double>(const double *f, int N, int c, int idx) {
    double2 v = reinterpret_cast<const double2 *>(f)[(size_t)c * N + idx];
    return Cx<double>{v.x, v.y};
}
template <>
__device__ __forceinline__ Cx<float> ld_cx<__nv_bfloat16, float>(const __nv_bfloat16 *f, int N, int c, int idx) {
    __nv_bfloat162 v = reinterpret_cast<const __nv_bfloat162 *>(f)[(size_t)c * N + idx];
    float2 w = __bfloat1622float2(v);
    return Cx<float>{w.x, w.y};
}
template <typename S, typename R>
__device__ __forceinline__ void st_cx(S *f, int N, int c, int idx, Cx<R> v);
template <>
__device__ __forceinline__ void st_cx<float, float>(float *f, int N, int c, int idx, Cx<float> v) {
    reinterpret_cast<float2 *>(f)[((size_t)(c >> 1) * N + idx) * 2 + (c & 1)] = make_float2(v.re, v.im);
}
template <>
__device__ __forceinline__ void st_cx<double, double>(double *f, int N, int c, int idx, Cx<double> v) {
    reinterpret_cast<double2 *>(f)[(size_t)c * N + idx] = make_double2(v.re, v.im);
}
template <>
__device__ __forceinline__ void st_cx<__nv_bfloat16, float>(__nv_bfloat16 *f, int N, int c, int idx, Cx<float> v) {
    reinterpret_cast<__nv_bfloat162 *>(f)[(size_t)c * N + idx] = __floats2bfloat162_rn(v.re, v.im);
}

// components (2k, 2k+1) of a spinor at one site: one 16-byte access for FP32
template <typename S, typename R>
__device__ __forceinline__ void ld_pair(const S *f, int N, int k, int idx, Cx<R> v[2]) {
    if constexpr (std::is_same<S, float>::value) {
        const float4 a = reinterpret_cast<const float4 *>(f)[(size_t)k * N + idx];
        v[0] = Cx<R>{a.x, a.y};
        v[1] = Cx<R>{a.z, a.w};
    } else {
        v[0] = ld_cx<S, R>(f, N, 2 * k, idx);
        v[1] = ld_cx<S, R>(f, N, 2 * k + 1, idx);
    }
}
template <typename S, typename R>
__device__ __forceinline__ void st_pair(S *f, int N, int k, int idx, const Cx<R> v[2]) {
    if constexpr (std::is_same<S, float>::value) {
        reinterpret_cast<float4 *>(f)[(size_t)k * N + idx] = make_float4(v[0].re, v[0].im, v[1].re, v[1].im);
    } else {
        st_cx<S, R>(f, N, 2 * k, idx, v[0]);
        st_cx<S, R>(f, N, 2 * k + 1, idx, v[1]);
    }
}

// whole spinor of one site, ps[spin][colour]: six 16-byte loads for FP32,
// twelve complex loads otherwise
template <typename S, typename R>
__device__ __forceinline__ void load_spinor(const S *f, int N, int idx, Cx<R> ps[4][3]) {
    if constexpr (std::is_same<S, float>::value) {
        const float4 *q = reinterpret_cast<const float4 *>(f);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 v = q[(size_t)k * N + idx];
            ps[(2 * k) / 3][(2 * k) % 3] = Cx<R>{v.x, v.y};
            ps[(2 * k + 1) / 3][(2 * k + 1) % 3] = Cx<R>{v.z, v.w};
        }
    } else {
#pragma unroll
        for (int c = 0; c < 12; ++c) ps[c / 3][c % 3] = ld_cx<S, R>(f, N, c, idx);
    }
}

template <typename S, typename R>
__device__ __forceinline__ void store_spinor(S *f, int N, int idx, const Cx<R> v[12]) {
    if constexpr (std::is_same<S, float>::value) {
        float4 *q = reinterpret_cast<float4 *>(f);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            q[(size_t)k * N + idx] = make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im);
    } else {
#pragma unroll
        for (int c = 0; c < 12; ++c) st_cx<S, R>(f, N, c, idx, v[c]);
    }
}

// ------------------------------------------------------------------ Wilson hop
// Spin projection in the chiral basis.  For direction mu and sg = -1 the
// projector is (1 - g_mu), for sg = +1 it is (1 + g_mu).  (1 -+ g_mu) psi is
// rebuilt from the half spinor h = (h0, h1) (two spins x 3 colours):
//   upper spins (0, 1) = (h0, h1), lower spins (2, 3) = L(h0, h1), with
//   mu = 0: h0 = p0 - sg i p3, h1 = p1 - sg i p2, L = ( sg i h1,  sg i h0)
//   mu = 1: h0 = p0 - sg p3,   h1 = p1 + sg p2,   L = ( sg h1,   -sg h0)
//   mu = 2: h0 = p0 - sg i p2, h1 = p1 + sg i p3, L = ( sg i h0, -sg i h1)
//   mu = 3: h0 = p0 + sg p2,   h1 = p1 + sg p3,   L = ( sg h0,    sg h1)
template <typename R>
__device__ __forceinline__ void spin_project(int mu, R sg, const Cx<R> ps[4][3], Cx<R> h[2][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Cx<R> p0 = ps[0][a], p1 = ps[1][a], p2 = ps[2][a], p3 = ps[3][a];
        if (mu == 0) {
            h[0][a] = csub(p0, cscale(ctimes_i(p3), sg));
            h[1][a] = csub(p1, cscale(ctimes_i(p2), sg));
        } else if (mu == 1) {
            h[0][a] = csub(p0, cscale(p3, sg));
            h[1][a] = cadd(p1, cscale(p2, sg));
        } else if (mu == 2) {
            h[0][a] = csub(p0, cscale(ctimes_i(p2), sg));
            h[1][a] = cadd(p1, cscale(ctimes_i(p3), sg));
        } else {
            h[0][a] = cadd(p0, cscale(p2, sg));
            h[1][a] = cadd(p1, cscale(p3, sg));
        }
    }
}

// v, or -v when n: the sign bit flipped on the integer pipe, the same bits as
// v * -1 without a floating-point multiply (FP64 issue slots are scarce)
__device__ __forceinline__ float neg_if(float v, bool n) { return __uint_as_float(__float_as_uint(v) ^ ((unsigned)n << 31)); }
__device__ __forceinline__ double neg_if(double v, bool n) {
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)((unsigned long long)n << 63));
}

// acc += eta * (rebuilt 4-spinor from the colour-rotated half spinor uh),
// eta = +1 or -1 (the boundary sign)
template <typename R>
__device__ __forceinline__ void spin_accumulate(int mu, R sg, R eta, const Cx<R> uh[2][3], Cx<R> acc[4][3]) {
    const bool neg = eta < R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const Cx<R> h0 = Cx<R>{neg_if(uh[0][a].re, neg), neg_if(uh[0][a].im, neg)};
        const Cx<R> h1 = Cx<R>{neg_if(uh[1][a].re, neg), neg_if(uh[1][a].im, neg)};
        acc[0][a] = cadd(acc[0][a], h0);
        acc[1][a] = cadd(acc[1][a], h1);
        if (mu == 0) {
            acc[2][a] = cadd(acc[2][a], cscale(ctimes_i(h1), sg));
            acc[3][a] = cadd(acc[3][a], cscale(ctimes_i(h0), sg));
        } else if (mu == 1) {
            acc[2][a] = cadd(acc[2][a], cscale(h1, sg));
            acc[3][a] = csub(acc[3][a], cscale(h0, sg));
        } else if (mu == 2) {
            acc[2][a] = cadd(acc[2][a], cscale(ctimes_i(h0), sg));
            acc[3][a] = csub(acc[3][a], cscale(ctimes_i(h1), sg));
        } else {
            acc[2][a] = cadd(acc[2][a], cscale(h0, sg));
            acc[3][a] = cadd(acc[3][a], cscale(h1, sg));
        }
    }
}

// links: complex [4][9][N] (FP64, BF16) or [4][5][N] 16-byte chunks (FP32)
template <typename R, typename LS>
__device__ __forceinline__ void load_link(const LS *U, int N, int mu, int idx, Cx<R> u[3][3]) {
    if constexpr (std::is_same<LS, float>::value) {
        const float4 *q = reinterpret_cast<const float4 *>(U) + (size_t)mu * 5 * N;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float4 v = q[(size_t)k * N + idx];
            u[(2 * k) / 3][(2 * k) % 3] = Cx<R>{v.x, v.y};
            if (k < 4) u[(2 * k + 1) / 3][(2 * k + 1) % 3] = Cx<R>{v.z, v.w};
        }
    } else {
#pragma unroll
        for (int e = 0; e < 9; ++e) u[e / 3][e % 3] = ld_cx<LS, R>(U, N, mu * 9 + e, idx);
    }
}

// ------------------------------------------------------------------ clover blocks
// The clover operator's site blocks 1 + C(x) and their inverses are, in the
// chiral basis, two Hermitian 6 x 6 blocks (components 6q .. 6q + 5 for
// chirality q; pt_op_set_clover packs them).  A block is 36 reals w: the six
// real diagonal entries, then the upper entries u_ij (i < j, row-major) as
// re, im; the lower entries are conj(u_ij).  v <- B v:
template <typename R>
__device__ __forceinline__ void herm6_mul(const R w[36], Cx<R> v[6]) {
    Cx<R> o[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) o[i] = cscale(v[i], w[i]);
    int k = 6;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i + 1; j < 6; ++j) {
            const Cx<R> u = Cx<R>{w[k], w[k + 1]};
            k += 2;
            o[i] = cadd(o[i], cmul(u, v[j]));
            o[j] = cadd(o[j], cconjmul(u, v[i]));
        }
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = o[i];
}

// v <- B v for the blocks of half entry h (Nh entries) in block array
// `which` of a packed clover array: FP32 chunks [which][18][Nh] float4, FP64
// [which][36][Nh] double2 (which 0: 1 + C on the even sites, 1: (1 + C)^{-1}
// on the odd ones, 2 (FP64 only): 1 + C on the odd ones)
__device__ __forceinline__ void clover_mul(const float4 *cl, int Nh, int which, int h, Cx<float> v[12]) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        float w[36];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float4 c = cl[((size_t)which * 18 + q * 9 + k) * Nh + h];
            w[4 * k] = c.x;
            w[4 * k + 1] = c.y;
            w[4 * k + 2] = c.z;
            w[4 * k + 3] = c.w;
        }
        herm6_mul<float>(w, v + 6 * q);
    }
}
__device__ __forceinline__ void clover_mul(const double2 *cl, int Nh, int which, int h, Cx<double> v[12]) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        double w[36];
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            const double2 c = cl[((size_t)which * 36 + q * 18 + k) * Nh + h];
            w[2 * k] = c.x;
            w[2 * k + 1] = c.y;
        }
        herm6_mul<double>(w, v + 6 * q);
    }
}

// (H psi)(x) for one site; psi is read through ld_cx from field f (N sites).
// Returns acc = H psi at x.
template <typename R, typename S, typename LS>
__device__ __forceinline__ void wilson_hop_site(const Geom &g, const S *f, const LS *U, int antip, int idx,
                                                const int x[4], Cx<R> acc[4][3]) {
    const int N = g.N;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[s][a] = Cx<R>{R(0), R(0)};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        // forward hop: (1 - g_mu) U_mu(x) psi(x + mu)
        {
            int y = nb_fwd(g, idx, x, mu);
            R eta = (antip && mu == 3 && x[3] == g.D[3] - 1) ? R(-1) : R(1);
            Cx<R> ps[4][3], h[2][3], uh[2][3], u[3][3];
            load_spinor<S, R>(f, N, y, ps);
            spin_project<R>(mu, R(-1), ps, h);
            load_link<R, LS>(U, N, mu, idx, u);
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Cx<R> t = cmul(u[a][0], h[k][0]);
                    t = cadd(t, cmul(u[a][1], h[k][1]));
                    t = cadd(t, cmul(u[a][2], h[k][2]));
                    uh[k][a] = t;
                }
            spin_accumulate<R>(mu, R(-1), eta, uh, acc);
        }
        // backward hop: (1 + g_mu) U_mu(x - mu)^dagger psi(x - mu)
        {
            int y = nb_bwd(g, idx, x, mu);
            R eta = (antip && mu == 3 && x[3] == 0) ? R(-1) : R(1);
            Cx<R> ps[4][3], h[2][3], uh[2][3], u[3][3];
            load_spinor<S, R>(f, N, y, ps);
            spin_project<R>(mu, R(1), ps, h);
            load_link<R, LS>(U, N, mu, y, u);
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    // (U^dagger h)_a = sum_b conj(U_ba) h_b
                    Cx<R> t = cconjmul(u[0][a], h[k][0]);
                    t = cadd(t, cconjmul(u[1][a], h[k][1]));
                    t = cadd(t, cconjmul(u[2][a], h[k][2]));
                    uh[k][a] = t;
                }
            spin_accumulate<R>(mu, R(1), eta, uh, acc);
        }
    }
}

// (H psi_n)(x) for NB right-hand sides at one site: every link is loaded once
// and applied to the NB spin-projected neighbours (the links of a site block
// are shared by the right-hand sides of the block).
template <typename R, typename S, typename LS, int NB>
__device__ __forceinline__ void wilson_hop_multi(const Geom &g, const S *const (&f)[NB], const LS *U, int antip,
                                                 int idx, const int x[4], Cx<R> (&acc)[NB][4][3]) {
    const int N = g.N;
#pragma unroll
    for (int n = 0; n < NB; ++n)
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[n][s][a] = Cx<R>{R(0), R(0)};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        {   // forward hop: (1 - g_mu) U_mu(x) psi(x + mu)
            const int y = nb_fwd(g, idx, x, mu);
            const R eta = (antip && mu == 3 && x[3] == g.D[3] - 1) ? R(-1) : R(1);
            Cx<R> u[3][3];
            load_link<R, LS>(U, N, mu, idx, u);
#pragma unroll
            for (int n = 0; n < NB; ++n) {
                Cx<R> ps[4][3], h[2][3], uh[2][3];
                load_spinor<S, R>(f[n], N, y, ps);
                spin_project<R>(mu, R(-1), ps, h);
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        Cx<R> t = cmul(u[a][0], h[k][0]);
                        t = cadd(t, cmul(u[a][1], h[k][1]));
                        t = cadd(t, cmul(u[a][2], h[k][2]));
                        uh[k][a] = t;
                    }
                spin_accumulate<R>(mu, R(-1), eta, uh, acc[n]);
            }
        }
        {   // backward hop: (1 + g_mu) U_mu(x - mu)^dagger psi(x - mu)
            const int y = nb_bwd(g, idx, x, mu);
            const R eta = (antip && mu == 3 && x[3] == 0) ? R(-1) : R(1);
            Cx<R> u[3][3];
            load_link<R, LS>(U, N, mu, y, u);
#pragma unroll
            for (int n = 0; n < NB; ++n) {
                Cx<R> ps[4][3], h[2][3], uh[2][3];
                load_spinor<S, R>(f[n], N, y, ps);
                spin_project<R>(mu, R(1), ps, h);
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        Cx<R> t = cconjmul(u[0][a], h[k][0]);
                        t = cadd(t, cconjmul(u[1][a], h[k][1]));
                        t = cadd(t, cconjmul(u[2][a], h[k][2]));
                        uh[k][a] = t;
                    }
                spin_accumulate<R>(mu, R(1), eta, uh, acc[n]);
            }
        }
    }
}

// Laplacian: (A f)(x) = (8 + m2) f(x) - sum_mu [f(x+mu) + f(x-mu)]
template <typename R, typename S>
__device__ __forceinline__ R lap_site(const Geom &g, const S *f, R diag, int idx, const int x[4]) {
    R nb = R(0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        nb += (R)ld_real(f, nb_fwd(g, idx, x, mu));
        nb += (R)ld_real(f, nb_bwd(g, idx, x, mu));
    }
    return diag * (R)ld_real(f, idx) - nb;
}

// ------------------------------------------------------------------ reductions
// Deterministic block sum of K doubles (fixed shuffle tree + fixed warp order).
// Result valid in thread 0.  `sh` needs 32 * K doubles.
template <int K>
__device__ __forceinline__ void block_sum(double v[K], double *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sh[warp * K + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[w * K + k];
            v[k] = s;
        }
    }
}

// ------------------------------------------------------------------ objects
struct pt_ctx {
    int device;
    cudaStream_t stream;
    cudaStream_t cap_stream;   // private stream used only to capture graphs (never executes work)
    cudaStream_t cap_side[2];  // side streams of a capture (branches of one engine iteration)
    cudaEvent_t cap_ev[3];     // fork / join markers of those branches
    bool own_stream;
    int num_sms;
    size_t mem_budget;
    int max_slots;           // 0: no cap on the right-hand sides in flight
    int64_t launch_limit;    // 0: the engine's own bound on graph launches per run
    // solver-engine parameters chosen by pt_autotune / pt_set_tuning, per
    // (operator kind, precision, lattice); `trial` overrides them while the
    // autotuner times a candidate
    struct Tune {
        int used, kind, prec, dims[4];
        double delta;
        int group, graph_iters, rhs_block, overlap, evenodd, cta_threads, sites_per_thread;
    } tune[16], trial;
    int in_trial;
    // grow-only work space
    void *ws;
    size_t ws_bytes;
    int *h_flags;            // pinned host mirror of device flags
    bool prof;
    int64_t prof_launches[4];
    double prof_ms[4];
};

struct pt_op {
    pt_ctx *ctx;
    int device;              // the context's device, kept so that pt_op_destroy never reads the context
    int kind;                // 0 Laplacian, 1 Wilson
    int dims[4];
    Geom g;
    int dof;
    double m2, kappa;
    int antip;
    double *U64;             // packed links complex [4][9][N], FP64
    float *U32;              // same, FP32
    __nv_bfloat16 *U16;      // same, BF16
    // clover term (pt_op_set_clover; Wilson, every side even): c_sw (0: none)
    // and the chiral 6 x 6 blocks of 1 + C per half-field entry, packed as 36
    // reals per chirality (clover_mul in engine.cu reads them):
    double csw;
    double *CL64;            // [3][36][N/2] double2: 1 + C even, (1 + C)^{-1} odd, 1 + C odd
    float *CL32;             // [2][18][N/2] float4: 1 + C even, (1 + C)^{-1} odd
};

// work-space helper: returns a device pointer of at least `bytes` (grow-only)
int pt_workspace(pt_ctx *ctx, size_t bytes, void **out);
int64_t pt_field_reals(const pt_op *op);   // L = N * dof * (1 or 2)

// kernels launched by the library (for launch counting)
extern thread_local int64_t pt_kernel_launch_count;
