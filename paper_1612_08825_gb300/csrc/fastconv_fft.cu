// FastConv by FFT for large kernels (Sec. IV-C, IV-D: above a kernel size threshold the
// FFT method is faster than the direct sum, and FastConv switches to it).
//
// Full convolution of extent M = N + K - 1 per axis: both operands are zero-padded to
// FFT sizes F >= M (products of 2, 3, 5 and 7), transformed real-to-complex with
// cuFFT, multiplied pointwise (with the 1 / prod(F) of the inverse), transformed back,
// and the M-extent corner is copied to the output.  Padding, the product and the crop
// are this file's kernels; the transforms are cuFFT's.  The plans belong to an explicit
// plan object (fastconv_fft_plan_create): they are made without an internal work area,
// and each call binds the work area inside the caller's workspace, so calls allocate
// nothing and calls on different streams never share scratch memory.
#include <cufft.h>

#include <algorithm>
#include <mutex>
#include <new>

#include "common.cuh"

namespace {

constexpr int kThreads = 256;

// smallest 2^a 3^b 5^c 7^d >= n
int64_t good_size(int64_t n)
{
    for (int64_t m = n;; ++m) {
        int64_t r = m;
        for (int f : {2, 3, 5, 7})
            while (r % f == 0) r /= f;
        if (r == 1) return m;
    }
}

struct Shape {
    int nd;
    int64_t F[3];          // FFT extents
    int64_t C;             // complex values: F[0..nd-2] x (F[nd-1] / 2 + 1)
    int64_t R;             // real values: prod(F)
};

Shape fft_shape(const int64_t *dims, int nd, const int64_t *kdims)
{
    Shape sh{};
    sh.nd = nd;
    sh.R = 1;
    sh.C = 1;
    for (int d = 0; d < nd; ++d) {
        sh.F[d] = good_size(dims[d] + kdims[d] - 1);
        sh.R *= sh.F[d];
        sh.C *= d + 1 < nd ? sh.F[d] : sh.F[d] / 2 + 1;
    }
    return sh;
}

struct Ext {
    int64_t a[3];           // extents, last fastest, unused leading ones 1
};

// dst (F extents, all R values) = src (N extents) zero-padded at the high end: block
// row blockIdx.y of the grid is destination row r = z * F1 + y; a block covers RSEG
// columns of it, four consecutive ones per thread (no divisions per element)
constexpr int RSEG = 4 * kThreads;

__global__ void __launch_bounds__(kThreads) pad_kernel(const float *__restrict__ src, Ext N, Ext F,
                                                       float *__restrict__ dst)
{
    const int64_t r = blockIdx.y + (int64_t)blockIdx.z * gridDim.y;
    if (r >= F.a[0] * F.a[1]) return;
    const int64_t z = r / F.a[1], y = r - z * F.a[1];
    const int64_t nx = (z < N.a[0] && y < N.a[1]) ? N.a[2] : 0;     // source columns of this row
    const float *s = src + (z * N.a[1] + y) * N.a[2];
    float *d = dst + r * F.a[2];
    const int64_t x0 = (int64_t)blockIdx.x * RSEG + threadIdx.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t x = x0 + k * kThreads;
        if (x < F.a[2]) d[x] = x < nx ? __ldg(s + x) : 0.f;
    }
}

// a[i] = a[i] * b[i] * scale
__global__ void __launch_bounds__(kThreads) mul_kernel(cufftComplex *__restrict__ a, const cufftComplex *__restrict__ b,
                                                       int64_t n, float scale)
{
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const cufftComplex u = a[i], v = b[i];
        a[i] = make_float2((u.x * v.x - u.y * v.y) * scale, (u.x * v.y + u.y * v.x) * scale);
    }
}

// out (M extents) = the M corner of src (F extents), one block row per output row, RSEG
// columns per block
__global__ void __launch_bounds__(kThreads) crop_kernel(const float *__restrict__ src, Ext F, Ext M,
                                                        float *__restrict__ out)
{
    const int64_t r = blockIdx.y + (int64_t)blockIdx.z * gridDim.y;
    if (r >= M.a[0] * M.a[1]) return;
    const int64_t z = r / M.a[1], y = r - z * M.a[1];
    const float *s = src + (z * F.a[1] + y) * F.a[2];
    float *o = out + r * M.a[2];
    const int64_t x0 = (int64_t)blockIdx.x * RSEG + threadIdx.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t x = x0 + k * kThreads;
        if (x < M.a[2]) o[x] = __ldg(s + x);
    }
}

Ext ext3(const int64_t *v, int nd)
{
    Ext e{{1, 1, 1}};
    for (int d = 0; d < nd; ++d) e.a[3 - nd + d] = v[d];
    return e;
}

unsigned grid_for(int64_t n)
{
    const int64_t b = ft::ceil_div(n, kThreads);
    return (unsigned)(b < 152 * 16 ? b : 152 * 16);
}

// grid for a row kernel: x over the columns (RSEG per block), y * z over the rows
dim3 row_grid(int64_t rows, int64_t cols)
{
    const int64_t bx = ft::ceil_div(cols, RSEG);
    const int64_t by = std::min<int64_t>(rows, 65535);
    const int64_t bz = ft::ceil_div(rows, by);
    return dim3((unsigned)bx, (unsigned)by, (unsigned)bz);
}

ft_status check_args(const int64_t *dims, int nd, const int64_t *kdims)
{
    if (!dims || !kdims) return FT_ERR_INVALID_ARG;
    if (nd < 1 || nd > FT_MAX_NDIM) return FT_ERR_SHAPE;
    for (int d = 0; d < nd; ++d)
        if (dims[d] < 1 || kdims[d] < 1) return FT_ERR_SHAPE;
    if (nd > 3) return FT_ERR_UNSUPPORTED;
    int64_t tot = 1;
    for (int d = 0; d < nd; ++d) {
        const int64_t m = dims[d] + kdims[d] - 1;
        if (m > (1 << 28) / 2) return FT_ERR_UNSUPPORTED;
        tot *= m;
        if (tot > ((int64_t)1 << 30)) return FT_ERR_UNSUPPORTED;
    }
    return FT_OK;
}

}  // namespace

struct fastconv_fft_plan {
    int dev;                  // the device the cuFFT plans were made on
    int nd;
    int64_t dims[3], kdims[3];
    Shape sh;
    cufftHandle fwd, inv;
    size_t pad_bytes;         // the two real and two complex arrays
    size_t work_bytes;        // cuFFT's work area (shared by the forward and inverse plans)
    std::mutex mu;            // serialises binding stream and work area + enqueueing
};

namespace {

// bytes of the padded real arrays and the complex spectra, each 256-byte aligned
void pad_sizes(const Shape &sh, size_t *r, size_t *c)
{
    *r = ((size_t)sh.R * sizeof(float) + 255) / 256 * 256;
    *c = ((size_t)sh.C * sizeof(cufftComplex) + 255) / 256 * 256;
}

}  // namespace

extern "C" ft_status fastconv_fft_plan_create(const int64_t *dims, int nd, const int64_t *kdims,
                                              fastconv_fft_plan **plan, size_t *workspace_bytes)
{
    FT_API_RANGE;
    if (!plan) return FT_ERR_INVALID_ARG;
    *plan = nullptr;
    const ft_status st = check_args(dims, nd, kdims);
    if (st != FT_OK) return st;
    fastconv_fft_plan *p = new (std::nothrow) fastconv_fft_plan();
    if (!p) return FT_ERR_CUDA;
    cudaError_t e = cudaGetDevice(&p->dev);
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        delete p;
        return FT_ERR_CUDA;
    }
    p->nd = nd;
    for (int d = 0; d < nd; ++d) {
        p->dims[d] = dims[d];
        p->kdims[d] = kdims[d];
    }
    p->sh = fft_shape(dims, nd, kdims);
    int n[3];
    for (int d = 0; d < nd; ++d) n[d] = (int)p->sh.F[d];
    size_t wf = 0, wi = 0;
    bool made_f = false, made_i = false;
    cufftResult r = cufftCreate(&p->fwd);
    if (r == CUFFT_SUCCESS) {
        made_f = true;
        r = cufftSetAutoAllocation(p->fwd, 0);
    }
    if (r == CUFFT_SUCCESS) r = cufftMakePlanMany(p->fwd, nd, n, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, 1, &wf);
    if (r == CUFFT_SUCCESS) r = cufftCreate(&p->inv);
    if (r == CUFFT_SUCCESS) {
        made_i = true;
        r = cufftSetAutoAllocation(p->inv, 0);
    }
    if (r == CUFFT_SUCCESS) r = cufftMakePlanMany(p->inv, nd, n, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 1, &wi);
    if (r != CUFFT_SUCCESS) {
        if (made_f) cufftDestroy(p->fwd);
        if (made_i) cufftDestroy(p->inv);
        delete p;
        ft::set_cuda_error(cudaErrorUnknown);
        return FT_ERR_CUDA;
    }
    size_t rb, cb;
    pad_sizes(p->sh, &rb, &cb);
    p->pad_bytes = 2 * rb + 2 * cb;
    p->work_bytes = (std::max(wf, wi) + 255) / 256 * 256;
    if (workspace_bytes) *workspace_bytes = p->pad_bytes + p->work_bytes;
    *plan = p;
    return FT_OK;
}

extern "C" void fastconv_fft_plan_destroy(fastconv_fft_plan *plan)
{
    if (!plan) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != plan->dev) cudaSetDevice(plan->dev);
    cufftDestroy(plan->fwd);
    cufftDestroy(plan->inv);
    if (cur != plan->dev) cudaSetDevice(cur);
    delete plan;
}

extern "C" size_t fastconv_fft_plan_workspace(const fastconv_fft_plan *plan)
{
    return plan ? plan->pad_bytes + plan->work_bytes : 0;
}

extern "C" ft_status fastconv_fft(fastconv_fft_plan *plan, const float *input, const float *kernel, float *out,
                                  void *workspace, size_t workspace_bytes, void *stream)
{
    FT_API_RANGE;
    if (!plan || !input || !kernel || !out || !workspace) return FT_ERR_INVALID_ARG;
    if (workspace_bytes < plan->pad_bytes + plan->work_bytes) return FT_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return FT_ERR_INVALID_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        ft::set_cuda_error(e);
        return FT_ERR_CUDA;
    }
    if (dev != plan->dev) return FT_ERR_INVALID_ARG;
    const int nd = plan->nd;
    const Shape &sh = plan->sh;
    size_t r, c;
    pad_sizes(sh, &r, &c);
    unsigned char *w = static_cast<unsigned char *>(workspace);
    float *ra = reinterpret_cast<float *>(w), *rb = reinterpret_cast<float *>(w + r);
    cufftComplex *ca = reinterpret_cast<cufftComplex *>(w + 2 * r);
    cufftComplex *cb = reinterpret_cast<cufftComplex *>(w + 2 * r + c);
    void *work = w + plan->pad_bytes;
    int64_t m[3];
    for (int d = 0; d < nd; ++d) m[d] = plan->dims[d] + plan->kdims[d] - 1;
    cudaStream_t s = ft::as_stream(stream);
    const Ext F = ext3(sh.F, nd);
    const dim3 pg = row_grid(F.a[0] * F.a[1], F.a[2]);
    pad_kernel<<<pg, kThreads, 0, s>>>(input, ext3(plan->dims, nd), F, ra);
    pad_kernel<<<pg, kThreads, 0, s>>>(kernel, ext3(plan->kdims, nd), F, rb);
    ft_status st = ft::check_launch();
    if (st != FT_OK) return st;
    {
        // the plans' stream and work area are bound per call; the lock keeps another
        // thread from rebinding them between this call's bind and its enqueue
        std::lock_guard<std::mutex> lock(plan->mu);
        cufftResult fr = cufftSetStream(plan->fwd, s);
        if (fr == CUFFT_SUCCESS) fr = cufftSetWorkArea(plan->fwd, work);
        if (fr == CUFFT_SUCCESS) fr = cufftExecR2C(plan->fwd, ra, ca);
        if (fr == CUFFT_SUCCESS) fr = cufftExecR2C(plan->fwd, rb, cb);
        if (fr == CUFFT_SUCCESS) {
            mul_kernel<<<grid_for(sh.C), kThreads, 0, s>>>(ca, cb, sh.C, (float)(1.0 / (double)sh.R));
            if ((st = ft::check_launch()) != FT_OK) return st;
            fr = cufftSetStream(plan->inv, s);
        }
        if (fr == CUFFT_SUCCESS) fr = cufftSetWorkArea(plan->inv, work);
        if (fr == CUFFT_SUCCESS) fr = cufftExecC2R(plan->inv, ca, ra);
        if (fr != CUFFT_SUCCESS) {
            ft::set_cuda_error(cudaErrorUnknown);
            return FT_ERR_CUDA;
        }
    }
    const Ext M = ext3(m, nd);
    crop_kernel<<<row_grid(M.a[0] * M.a[1], M.a[2]), kThreads, 0, s>>>(ra, F, M, out);
    return ft::check_launch();
}

// The switch to the FFT path: measured on GB300 for 2-D 1080 x 1920 images (the
// crossover sweep of the bench), so only 2-D requests of at least that output area
// with at least FT_FFT_MIN_TAPS taps take it; 3-D kernels and small images, whose
// crossover was not measured, stay on the direct path (with its per-element bound).
extern "C" int fastconv_prefers_fft(const int64_t *dims, int nd, const int64_t *kdims)
{
    if (check_args(dims, nd, kdims) != FT_OK || nd != 2) return 0;
    const int64_t taps = kdims[0] * kdims[1];
    const int64_t area = (dims[0] + kdims[0] - 1) * (dims[1] + kdims[1] - 1);
    return taps >= FT_FFT_MIN_TAPS && area >= FT_FFT_MIN_OUTPUT ? 1 : 0;
}
