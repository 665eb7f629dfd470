// Context, operators, errors, layout conversion, probes and the plain apply.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "pt_common.cuh"

thread_local int64_t pt_kernel_launch_count = 0;
static thread_local char g_err[512] = "";

void pt_set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int pt_cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    pt_set_error("CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e), cudaGetErrorString(e), what, file,
                 line);
    return e == cudaErrorMemoryAllocation ? PT_ERR_OOM : PT_ERR_CUDA;
}

extern "C" int pt_version(void) { return 100; }

extern "C" int pt_last_error(char *buf, size_t n) {
    if (!buf || n == 0) return PT_ERR_ARG;
    strncpy(buf, g_err, n - 1);
    buf[n - 1] = 0;
    return PT_OK;
}

extern "C" int pt_create(pt_ctx **out, int device, void *stream) {
    PT_CHECK_ARG(out != nullptr, "pt_create: ctx is NULL");
    *out = nullptr;
    int ndev = 0;
    PT_CUDA(cudaGetDeviceCount(&ndev));
    PT_CHECK_ARG(device >= 0 && device < ndev, "pt_create: device %d out of range (%d devices)", device, ndev);
    PT_CUDA(cudaSetDevice(device));
    pt_ctx *c = (pt_ctx *)calloc(1, sizeof(pt_ctx));
    if (!c) { pt_set_error("pt_create: host allocation failed"); return PT_ERR_OOM; }
    c->device = device;
    c->mem_budget = (size_t)16 << 30;
    if (stream) {
        c->stream = (cudaStream_t)stream;
        c->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { free(c); return pt_cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__); }
        c->own_stream = true;
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = cudaMallocHost((void **)&c->h_flags, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&c->cap_side[i], cudaStreamNonBlocking);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&c->cap_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (c->h_flags) cudaFreeHost(c->h_flags);
        if (c->own_stream) cudaStreamDestroy(c->stream);
        free(c);
        return pt_cuda_fail(e, "pt_create", __FILE__, __LINE__);
    }
    *out = c;
    return PT_OK;
}

extern "C" int pt_destroy(pt_ctx *c) {
    if (!c) return PT_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->ws) cudaFree(c->ws);
    if (c->h_flags) cudaFreeHost(c->h_flags);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (int i = 0; i < 2; ++i) if (c->cap_side[i]) cudaStreamDestroy(c->cap_side[i]);
    for (int i = 0; i < 3; ++i) if (c->cap_ev[i]) cudaEventDestroy(c->cap_ev[i]);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    free(c);
    return PT_OK;
}

extern "C" int pt_synchronize(pt_ctx *c) {
    PT_CHECK_ARG(c, "pt_synchronize: ctx is NULL");
    PT_CUDA(cudaStreamSynchronize(c->stream));
    return PT_OK;
}

extern "C" int pt_set_memory_budget(pt_ctx *c, size_t bytes) {
    PT_CHECK_ARG(c && bytes >= ((size_t)1 << 24), "pt_set_memory_budget: budget below 16 MiB");
    c->mem_budget = bytes;
    return PT_OK;
}

extern "C" int pt_set_max_slots(pt_ctx *c, int n) {
    PT_CHECK_ARG(c && n >= 0, "pt_set_max_slots: need n >= 0");
    c->max_slots = n;
    return PT_OK;
}

extern "C" int pt_set_launch_limit(pt_ctx *c, int64_t n) {
    PT_CHECK_ARG(c && n >= 0, "pt_set_launch_limit: need n >= 0");
    c->launch_limit = n;
    return PT_OK;
}

extern "C" int pt_profile_enable(pt_ctx *c, int on) {
    PT_CHECK_ARG(c, "pt_profile_enable: ctx is NULL");
    c->prof = on != 0;
    return PT_OK;
}

extern "C" int pt_profile_read(pt_ctx *c, int which, int64_t *launches, double *ms, int reset) {
    PT_CHECK_ARG(c && which >= 0 && which < 4, "pt_profile_read: bad arguments");
    if (launches) *launches = c->prof_launches[which];
    if (ms) *ms = c->prof_ms[which];
    if (reset) { c->prof_launches[which] = 0; c->prof_ms[which] = 0.0; }
    return PT_OK;
}

int pt_workspace(pt_ctx *c, size_t bytes, void **out) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes > c->ws_bytes) {
        cudaStreamSynchronize(c->stream);
        if (c->ws) { cudaFree(c->ws); c->ws = nullptr; c->ws_bytes = 0; }
        cudaError_t e = cudaMalloc(&c->ws, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            pt_set_error("work space allocation of %zu bytes failed (%s)", bytes, cudaGetErrorString(e));
            return PT_ERR_OOM;
        }
        c->ws_bytes = bytes;
    }
    *out = c->ws;
    return PT_OK;
}

int64_t pt_field_reals(const pt_op *op) { return (int64_t)op->g.N * (op->dof == 1 ? 1 : 24); }

static int check_dims(const int dims[4]) {
    if (!dims) return 0;
    int64_t n = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 1 || dims[mu] > (1 << 20)) return 0;
        n *= dims[mu];
    }
    return n <= ((int64_t)1 << 30);
}

// ------------------------------------------------------------------ link packing
// user [N][4][3][3] complex128 -> packed complex [4][9][N] in FP64 and BF16,
// and [4][5][N] 16-byte chunks (entries 2k, 2k+1) in FP32
__global__ void k_pack_links(int N, const double2 *__restrict__ Uu, double2 *U64, float2 *U32,
                             __nv_bfloat162 *U16) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)N * 36) return;
    int idx = (int)(i / 36), r = (int)(i % 36);   // r = mu * 9 + e
    double2 v = Uu[i];
    int64_t o = (int64_t)r * N + idx;
    U64[o] = v;
    const int mu = r / 9, el = r % 9;
    U32[(((int64_t)mu * 5 + el / 2) * N + idx) * 2 + (el & 1)] = make_float2((float)v.x, (float)v.y);
    U16[o] = __floats2bfloat162_rn((float)v.x, (float)v.y);
}

extern "C" int pt_op_laplacian(pt_ctx *c, const int dims[4], double m2, pt_op **out) {
    PT_CHECK_ARG(c && out, "pt_op_laplacian: NULL argument");
    PT_CHECK_ARG(check_dims(dims), "pt_op_laplacian: invalid lattice dimensions");
    pt_op *op = (pt_op *)calloc(1, sizeof(pt_op));
    if (!op) { pt_set_error("host allocation failed"); return PT_ERR_OOM; }
    op->ctx = c;
    op->device = c->device;
    op->kind = 0;
    memcpy(op->dims, dims, 4 * sizeof(int));
    op->g = make_geom(dims);
    op->dof = 1;
    op->m2 = m2;
    *out = op;
    return PT_OK;
}

extern "C" int pt_op_wilson(pt_ctx *c, const int dims[4], const double *U_dev, double kappa, int antip,
                            pt_op **out) {
    PT_CHECK_ARG(c && out && U_dev, "pt_op_wilson: NULL argument");
    PT_CHECK_ARG(check_dims(dims), "pt_op_wilson: invalid lattice dimensions");
    PT_CUDA(cudaSetDevice(c->device));
    pt_op *op = (pt_op *)calloc(1, sizeof(pt_op));
    if (!op) { pt_set_error("host allocation failed"); return PT_ERR_OOM; }
    op->ctx = c;
    op->device = c->device;
    op->kind = 1;
    memcpy(op->dims, dims, 4 * sizeof(int));
    op->g = make_geom(dims);
    op->dof = 12;
    op->kappa = kappa;
    op->antip = antip ? 1 : 0;
    size_t n = (size_t)op->g.N * 36;
    cudaError_t e = cudaMalloc((void **)&op->U64, n * sizeof(double2));
    // FP32 links: [4][5][N] 16-byte chunks (9 complex entries + 1 zero pad per link)
    if (e == cudaSuccess) e = cudaMalloc((void **)&op->U32, (size_t)op->g.N * 20 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc((void **)&op->U16, n * sizeof(__nv_bfloat162));
    if (e != cudaSuccess) {
        cudaFree(op->U64); cudaFree(op->U32); cudaFree(op->U16); free(op);
        cudaGetLastError();
        pt_set_error("pt_op_wilson: link allocation failed (%s)", cudaGetErrorString(e));
        return PT_ERR_OOM;
    }
    int threads = 256;
    int64_t blocks = ((int64_t)n + threads - 1) / threads;
    e = cudaMemsetAsync(op->U32, 0, (size_t)op->g.N * 20 * sizeof(float4), c->stream);   // pad entries
    if (e != cudaSuccess) { cudaFree(op->U64); cudaFree(op->U32); cudaFree(op->U16); free(op);
                            return pt_cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__); }
    k_pack_links<<<(unsigned)blocks, threads, 0, c->stream>>>(op->g.N, (const double2 *)U_dev,
                                                               (double2 *)op->U64, (float2 *)op->U32,
                                                               (__nv_bfloat162 *)op->U16);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    *out = op;
    return PT_OK;
}

extern "C" int pt_op_dof(const pt_op *op) { return op ? op->dof : PT_ERR_ARG; }

// Does not read the context: an operator may outlive it (a garbage collector
// finalises objects of a reference cycle in no particular order).  cudaFree
// waits for the device, so no work that still reads the links is cut short.
extern "C" int pt_op_destroy(pt_op *op) {
    if (!op) return PT_OK;
    if (op->kind == 1) {
        cudaSetDevice(op->device);
        cudaFree(op->U64); cudaFree(op->U32); cudaFree(op->U16);
        cudaFree(op->CL64); cudaFree(op->CL32);
    }
    free(op);
    return PT_OK;
}

// ------------------------------------------------------------------ layout conversion
// user [nrhs][N][12] complex128  <->  internal [nrhs][12][N] complex (precision S)
template <typename S>
__global__ void k_user_to_internal(int N, int dof, int nrhs, const double *__restrict__ in, S *out) {
    typedef typename ArithT<S>::T R;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)nrhs * N * dof;
    if (i >= tot) return;
    if (dof == 1) { st_real(out, (size_t)i, (R)in[i]); return; }
    int64_t j = i / ((int64_t)N * 12);
    int64_t r = i % ((int64_t)N * 12);
    int c = (int)(r / N), idx = (int)(r % N);               // internal order: component-major
    const double *src = in + ((j * N + idx) * 12 + c) * 2;
    st_cx<S, R>(out + (size_t)j * 24 * N, N, c, idx, Cx<R>{(R)src[0], (R)src[1]});
}

template <typename S>
__global__ void k_internal_to_user(int N, int dof, int nrhs, const S *__restrict__ in, double *out) {
    typedef typename ArithT<S>::T R;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)nrhs * N * dof;
    if (i >= tot) return;
    if (dof == 1) { out[i] = (double)ld_real(in, (size_t)i); return; }
    int64_t j = i / ((int64_t)N * 12);
    int64_t r = i % ((int64_t)N * 12);
    int c = (int)(r / N), idx = (int)(r % N);
    Cx<R> v = ld_cx<S, R>(in + (size_t)j * 24 * N, N, c, idx);
    double *dst = out + ((j * N + idx) * 12 + c) * 2;
    dst[0] = (double)v.re;
    dst[1] = (double)v.im;
}

template <typename S>
int launch_user_to_internal(pt_ctx *c, int N, int dof, int nrhs, const double *in, S *out) {
    int64_t tot = (int64_t)nrhs * N * dof;
    if (tot == 0) return PT_OK;
    k_user_to_internal<S><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(N, dof, nrhs, in, out);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    return PT_OK;
}
template <typename S>
int launch_internal_to_user(pt_ctx *c, int N, int dof, int nrhs, const S *in, double *out) {
    int64_t tot = (int64_t)nrhs * N * dof;
    if (tot == 0) return PT_OK;
    k_internal_to_user<S><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(N, dof, nrhs, in, out);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    return PT_OK;
}
template int launch_user_to_internal<double>(pt_ctx *, int, int, int, const double *, double *);
template int launch_internal_to_user<double>(pt_ctx *, int, int, int, const double *, double *);

// ------------------------------------------------------------------ plain apply
// one thread per (site, rhs); y = A x in the internal layout
template <typename R, typename S, typename LS>
__global__ void k_apply(Geom g, int kind, int nrhs, R diag, R kappa, int antip, const LS *__restrict__ U,
                        const S *__restrict__ x, S *__restrict__ y) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (idx >= g.N || j >= nrhs) return;
    int xc[4];
    site_coords(g, idx, xc);
    if (kind == 0) {
        const S *xj = x + (size_t)j * g.N;
        R v = lap_site<R, S>(g, xj, diag, idx, xc);
        st_real(y + (size_t)j * g.N, idx, v);
    } else {
        const S *xj = x + (size_t)j * 24 * g.N;
        S *yj = y + (size_t)j * 24 * g.N;
        Cx<R> acc[4][3];
        wilson_hop_site<R, S, LS>(g, xj, U, antip, idx, xc, acc);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                Cx<R> v = ld_cx<S, R>(xj, g.N, 3 * s + a, idx);
                st_cx<S, R>(yj, g.N, 3 * s + a, idx, csub(v, cscale(acc[s][a], kappa)));
            }
    }
}

template <typename R, typename S, typename LS>
static int apply_prec(const pt_op *op, const double *x_dev, double *y_dev, int nrhs, const LS *U) {
    pt_ctx *c = op->ctx;
    const int N = op->g.N;
    const size_t L = (size_t)pt_field_reals(op);
    void *ws;
    int rc = pt_workspace(c, 2 * (size_t)nrhs * L * sizeof(S), &ws);
    if (rc) return rc;
    S *xi = (S *)ws, *yi = xi + (size_t)nrhs * L;
    if ((rc = launch_user_to_internal<S>(c, N, op->dof, nrhs, x_dev, xi))) return rc;
    dim3 grid((N + 127) / 128, nrhs);
    k_apply<R, S, LS><<<grid, 128, 0, c->stream>>>(op->g, op->kind, nrhs, (R)(8.0 + op->m2), (R)op->kappa,
                                                     op->antip, U, xi, yi);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    return launch_internal_to_user<S>(c, N, op->dof, nrhs, yi, y_dev);
}

template int launch_user_to_internal<float>(pt_ctx *, int, int, int, const double *, float *);
template int launch_internal_to_user<float>(pt_ctx *, int, int, int, const float *, double *);
template int launch_user_to_internal<__nv_bfloat16>(pt_ctx *, int, int, int, const double *, __nv_bfloat16 *);
template int launch_internal_to_user<__nv_bfloat16>(pt_ctx *, int, int, int, const __nv_bfloat16 *, double *);

// y += C x for a clover operator (user layout, FP64): C = (1 + C) - 1 with
// the packed blocks 1 + C (even sites: array 0, odd sites: array 2)
__global__ void k_clover_add(Geom g, const double2 *CL64, const double *x, double *y, int nrhs) {
    const int N = g.N;
    const int64_t total = (int64_t)nrhs * N;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(t % N);
        int xc[4];
        site_coords(g, s, xc);
        const int par = (xc[0] + xc[1] + xc[2] + xc[3]) & 1;
        const double *xv = x + (size_t)t * 24;
        double *yv = y + (size_t)t * 24;
        Cx<double> v[12];
        for (int c = 0; c < 12; ++c) v[c] = Cx<double>{xv[2 * c], xv[2 * c + 1]};
        clover_mul(CL64, N / 2, par ? 2 : 0, s >> 1, v);
        for (int c = 0; c < 12; ++c) {
            yv[2 * c] += v[c].re - xv[2 * c];
            yv[2 * c + 1] += v[c].im - xv[2 * c + 1];
        }
    }
}

extern "C" int pt_apply(pt_ctx *c, const pt_op *op, const double *x_dev, double *y_dev, int nrhs, int prec) {
    PT_CHECK_ARG(c && op && op->ctx == c, "pt_apply: bad context/operator");
    PT_CHECK_ARG(nrhs >= 0 && nrhs <= 65535, "pt_apply: nrhs must be in [0, 65535]");
    if (nrhs == 0) return PT_OK;
    PT_CHECK_ARG(x_dev && y_dev && x_dev != y_dev, "pt_apply: NULL or aliased fields");
    PT_CUDA(cudaSetDevice(c->device));
    int rc;
    switch (prec) {
        case PT_PREC_FP64: rc = apply_prec<double, double, double>(op, x_dev, y_dev, nrhs, op->U64); break;
        case PT_PREC_MIXED_FP32: rc = apply_prec<float, float, float>(op, x_dev, y_dev, nrhs, op->U32); break;
        case PT_PREC_MIXED_BF16:
            rc = apply_prec<float, __nv_bfloat16, __nv_bfloat16>(op, x_dev, y_dev, nrhs, op->U16);
            break;
        default: PT_CHECK_ARG(false, "pt_apply: unknown precision %d", prec);
    }
    if (rc != PT_OK || op->csw == 0.0) return rc;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)nrhs * op->g.N + 127) / 128,
                                                                  16 * c->num_sms));
    k_clover_add<<<grid, 128, 0, c->stream>>>(op->g, (const double2 *)op->CL64, x_dev, y_dev, nrhs);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    return PT_OK;
}

// ------------------------------------------------------------------ probes
__global__ void k_make_probe(int64_t N, const int32_t *__restrict__ col, int colour, int kind, uint64_t key,
                             int dof, int comp, double *v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    bool on = col[i] == colour;
    if (dof == 1) {
        v[i] = on ? pt_noise(key, (uint64_t)i, kind).re : 0.0;
        return;
    }
    for (int a = 0; a < 12; ++a) {
        Cx<double> z = {0.0, 0.0};
        if (on) {
            if (comp < 0) z = pt_noise(key, (uint64_t)i * 12 + a, kind);       // undiluted
            else if (a == comp) z = pt_noise(key, (uint64_t)i, kind);          // diluted
        }
        v[(i * 12 + a) * 2] = z.re;
        v[(i * 12 + a) * 2 + 1] = z.im;
    }
}

extern "C" int pt_make_probes(pt_ctx *c, const int32_t *col_dev, int64_t N, int colour, int noise, uint64_t seed,
                              int set, int dof, int component, double *v_dev) {
    PT_CHECK_ARG(c && col_dev && v_dev && N > 0, "pt_make_probes: NULL argument or N <= 0");
    PT_CHECK_ARG(dof == 1 || dof == 12, "pt_make_probes: dof must be 1 or 12");
    PT_CHECK_ARG(noise == PT_NOISE_Z2 || (noise == PT_NOISE_Z4 && dof == 12),
                 "pt_make_probes: Z4 noise needs a complex (dof 12) field");
    PT_CHECK_ARG(component >= -1 && component < dof, "pt_make_probes: component out of range");
    PT_CUDA(cudaSetDevice(c->device));
    k_make_probe<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(N, col_dev, colour, noise,
                                                                        pt_set_key(seed, set), dof, component, v_dev);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    return PT_OK;
}
