// Vector operations of the building-block Krylov solvers, with one interface
// on the device (kernels on the context stream; dot products summed in a
// fixed order) and on the host (plain loops), so that a solver written once
// as a template over the executor runs on either.
#pragma once

#include <vector>

#include "hd_complex.cuh"
#include "pt_common.cuh"

// vector operations on n reals (complex fields: interleaved pairs)
static __global__ void k_vec_axpy(long n, int cplx, double ar, double ai, const double *x, double *y) {
    const long m = cplx ? n / 2 : n;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long)gridDim.x * blockDim.x) {
        if (cplx) {
            const double xr = x[2 * t], xi = x[2 * t + 1];
            y[2 * t] += ar * xr - ai * xi;
            y[2 * t + 1] += ar * xi + ai * xr;
        } else {
            y[t] += ar * x[t];
        }
    }
}
static __global__ void k_vec_xpay(long n, int cplx, const double *x, double br, double bi, double *y) {
    const long m = cplx ? n / 2 : n;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long)gridDim.x * blockDim.x) {
        if (cplx) {
            const double yr = y[2 * t], yi = y[2 * t + 1];
            y[2 * t] = x[2 * t] + br * yr - bi * yi;
            y[2 * t + 1] = x[2 * t + 1] + br * yi + bi * yr;
        } else {
            y[t] = x[t] + br * y[t];
        }
    }
}
// partials[block] = sum over the block's elements of conj(x) y, in a fixed order
#define VEC_DOT_BLOCKS 256
static __global__ void __launch_bounds__(256) k_vec_dot(long n, int cplx, const double *x, const double *y,
                                                double *partials) {
    __shared__ double sh[2][8];
    const long m = cplx ? n / 2 : n;
    double re = 0.0, im = 0.0;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long)gridDim.x * blockDim.x) {
        if (cplx) {
            const double xr = x[2 * t], xi = x[2 * t + 1], yr = y[2 * t], yi = y[2 * t + 1];
            re += xr * yr + xi * yi;
            im += xr * yi - xi * yr;
        } else {
            re += x[t] * y[t];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sh[0][warp] = re; sh[1][warp] = im; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) { a += sh[0][w]; b += sh[1][w]; }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

struct DevVec {
    pt_ctx *c = nullptr;
    double *dot_part = nullptr;   // VEC_DOT_BLOCKS complex partials (allocated by the solver)
    std::vector<double> h_part;
    double *alloc(size_t n) {
        double *p = nullptr;
        if (cudaMallocAsync((void **)&p, n * sizeof(double), c->stream) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void release(double *p) { cudaFreeAsync(p, c->stream); }
    int vgrid(long m) const { return (int)std::max(1L, std::min((m + 255) / 256, 16L * c->num_sms)); }
    int axpy(long n, int cplx, zd a, const double *x, double *y) {
        k_vec_axpy<<<vgrid(cplx ? n / 2 : n), 256, 0, c->stream>>>(n, cplx, a.re, a.im, x, y);
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
        return PT_OK;
    }
    int xpay(long n, int cplx, const double *x, zd b, double *y) {
        k_vec_xpay<<<vgrid(cplx ? n / 2 : n), 256, 0, c->stream>>>(n, cplx, x, b.re, b.im, y);
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
        return PT_OK;
    }
    int copy(long n, const double *x, double *y) {
        PT_CUDA(cudaMemcpyAsync(y, x, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        return PT_OK;
    }
    int zero(long n, double *y) {
        PT_CUDA(cudaMemsetAsync(y, 0, (size_t)n * sizeof(double), c->stream));
        return PT_OK;
    }
    int dot(long n, int cplx, const double *x, const double *y, zd *out) {
        k_vec_dot<<<VEC_DOT_BLOCKS, 256, 0, c->stream>>>(n, cplx, x, y, dot_part);
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
        h_part.resize(2 * VEC_DOT_BLOCKS);
        PT_CUDA(cudaMemcpyAsync(h_part.data(), dot_part, h_part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
        PT_CUDA(cudaStreamSynchronize(c->stream));
        zd acc = {0.0, 0.0};
        for (int k = 0; k < VEC_DOT_BLOCKS; ++k) acc = zadd(acc, zd{h_part[2 * k], h_part[2 * k + 1]});
        *out = acc;
        return PT_OK;
    }
};

struct HostVec {
    pt_ctx *c = nullptr;          // unused on the host
    double *dot_part = nullptr;   // unused on the host
    std::vector<std::vector<double>> bufs;
    double *alloc(size_t n) {
        bufs.emplace_back(n, 0.0);
        return bufs.back().data();
    }
    void release(double *p) {
        for (size_t k = 0; k < bufs.size(); ++k)
            if (bufs[k].data() == p) { bufs.erase(bufs.begin() + (long)k); return; }
    }
    int axpy(long n, int cplx, zd a, const double *x, double *y) {
        if (cplx)
            for (long t = 0; t < n / 2; ++t) {
                const zd v = zadd(zd{y[2 * t], y[2 * t + 1]}, zmulc(a, zd{x[2 * t], x[2 * t + 1]}));
                y[2 * t] = v.re;
                y[2 * t + 1] = v.im;
            }
        else
            for (long t = 0; t < n; ++t) y[t] += a.re * x[t];
        return PT_OK;
    }
    int xpay(long n, int cplx, const double *x, zd b, double *y) {
        if (cplx)
            for (long t = 0; t < n / 2; ++t) {
                const zd v = zadd(zd{x[2 * t], x[2 * t + 1]}, zmulc(b, zd{y[2 * t], y[2 * t + 1]}));
                y[2 * t] = v.re;
                y[2 * t + 1] = v.im;
            }
        else
            for (long t = 0; t < n; ++t) y[t] = x[t] + b.re * y[t];
        return PT_OK;
    }
    int copy(long n, const double *x, double *y) {
        for (long t = 0; t < n; ++t) y[t] = x[t];
        return PT_OK;
    }
    int zero(long n, double *y) {
        for (long t = 0; t < n; ++t) y[t] = 0.0;
        return PT_OK;
    }
    int dot(long n, int cplx, const double *x, const double *y, zd *out) {
        zd acc = {0.0, 0.0};
        if (cplx)
            for (long t = 0; t < n / 2; ++t)
                acc = zadd(acc, zmulc(zconj(zd{x[2 * t], x[2 * t + 1]}), zd{y[2 * t], y[2 * t + 1]}));
        else
            for (long t = 0; t < n; ++t) acc.re += x[t] * y[t];
        *out = acc;
        return PT_OK;
    }
};
