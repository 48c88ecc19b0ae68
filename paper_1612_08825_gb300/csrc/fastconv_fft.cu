// FastConv by FFT for large kernels (Sec. IV-C, IV-D: above a kernel size threshold the
// FFT method is faster than the direct sum, and FastConv switches to it).
//
// Full convolution of extent M = N + K - 1 per axis: both operands are zero-padded to
// FFT sizes F >= M (products of 2, 3, 5 and 7), transformed real-to-complex with
// cuFFT, multiplied pointwise (with the 1 / prod(F) of the inverse), transformed back,
// and the M-extent corner is copied to the output.  Padding, the product and the crop
// are this file's kernels; the transforms are cuFFT's, with plans cached per shape.
#include <cufft.h>

#include <algorithm>

#include <map>
#include <mutex>
#include <vector>

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

struct Plans {
    cufftHandle fwd, inv;
};

std::mutex g_mu;
std::map<std::vector<int64_t>, Plans> g_plans;   // key: device, F[0..nd-1]

cufftResult get_plans(const Shape &sh, Plans *out)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<int64_t> key{dev};
    for (int d = 0; d < sh.nd; ++d) key.push_back(sh.F[d]);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
        *out = it->second;
        return CUFFT_SUCCESS;
    }
    int n[3];
    for (int d = 0; d < sh.nd; ++d) n[d] = (int)sh.F[d];
    Plans p{};
    cufftResult r = cufftPlanMany(&p.fwd, sh.nd, n, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, 1);
    if (r != CUFFT_SUCCESS) return r;
    r = cufftPlanMany(&p.inv, sh.nd, n, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 1);
    if (r != CUFFT_SUCCESS) {
        cufftDestroy(p.fwd);
        return r;
    }
    g_plans[key] = p;
    *out = p;
    return CUFFT_SUCCESS;
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

extern "C" ft_status fastconv_fft_workspace(const int64_t *dims, int nd, const int64_t *kdims, size_t *bytes)
{
    if (!bytes) return FT_ERR_INVALID_ARG;
    const ft_status st = check_args(dims, nd, kdims);
    if (st != FT_OK) return st;
    const Shape sh = fft_shape(dims, nd, kdims);
    // two real arrays and two complex arrays, each 256-byte aligned
    const size_t r = ((size_t)sh.R * sizeof(float) + 255) / 256 * 256;
    const size_t c = ((size_t)sh.C * sizeof(cufftComplex) + 255) / 256 * 256;
    *bytes = 2 * r + 2 * c;
    return FT_OK;
}

extern "C" ft_status fastconv_fft(const float *input, const int64_t *dims, int nd, const float *kernel,
                                  const int64_t *kdims, float *out, void *workspace, size_t workspace_bytes,
                                  void *stream)
{
    if (!input || !kernel || !out || !workspace) return FT_ERR_INVALID_ARG;
    ft_status st = check_args(dims, nd, kdims);
    if (st != FT_OK) return st;
    size_t need = 0;
    fastconv_fft_workspace(dims, nd, kdims, &need);
    if (workspace_bytes < need) return FT_ERR_WORKSPACE;
    const Shape sh = fft_shape(dims, nd, kdims);
    const size_t r = ((size_t)sh.R * sizeof(float) + 255) / 256 * 256;
    const size_t c = ((size_t)sh.C * sizeof(cufftComplex) + 255) / 256 * 256;
    unsigned char *w = static_cast<unsigned char *>(workspace);
    float *ra = reinterpret_cast<float *>(w), *rb = reinterpret_cast<float *>(w + r);
    cufftComplex *ca = reinterpret_cast<cufftComplex *>(w + 2 * r);
    cufftComplex *cb = reinterpret_cast<cufftComplex *>(w + 2 * r + c);
    int64_t m[3];
    int64_t mtot = 1;
    for (int d = 0; d < nd; ++d) {
        m[d] = dims[d] + kdims[d] - 1;
        mtot *= m[d];
    }
    cudaStream_t s = ft::as_stream(stream);
    const Ext F = ext3(sh.F, nd);
    const dim3 pg = row_grid(F.a[0] * F.a[1], F.a[2]);
    pad_kernel<<<pg, kThreads, 0, s>>>(input, ext3(dims, nd), F, ra);
    pad_kernel<<<pg, kThreads, 0, s>>>(kernel, ext3(kdims, nd), F, rb);
    if ((st = ft::check_launch()) != FT_OK) return st;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        Plans p;
        cufftResult fr = get_plans(sh, &p);
        if (fr == CUFFT_SUCCESS) fr = cufftSetStream(p.fwd, s);
        if (fr == CUFFT_SUCCESS) fr = cufftSetStream(p.inv, s);
        if (fr == CUFFT_SUCCESS) fr = cufftExecR2C(p.fwd, ra, ca);
        if (fr == CUFFT_SUCCESS) fr = cufftExecR2C(p.fwd, rb, cb);
        if (fr == CUFFT_SUCCESS) {
            mul_kernel<<<grid_for(sh.C), kThreads, 0, s>>>(ca, cb, sh.C, (float)(1.0 / (double)sh.R));
            if ((st = ft::check_launch()) != FT_OK) return st;
            fr = cufftExecC2R(p.inv, ca, ra);
        }
        if (fr != CUFFT_SUCCESS) {
            ft::set_cuda_error(cudaErrorUnknown);
            return FT_ERR_CUDA;
        }
    }
    const Ext M = ext3(m, nd);
    crop_kernel<<<row_grid(M.a[0] * M.a[1], M.a[2]), kThreads, 0, s>>>(ra, F, M, out);
    return ft::check_launch();
}

// The kernel size above which the FFT path is faster on this part (measured with the
// bench's crossover sweep on 1080 x 1920 images: see FT_FFT_MIN_TAPS in the header).
extern "C" int fastconv_prefers_fft(const int64_t *dims, int nd, const int64_t *kdims)
{
    if (check_args(dims, nd, kdims) != FT_OK) return 0;
    int64_t taps = 1;
    for (int d = 0; d < nd; ++d) taps *= kdims[d];
    return taps >= FT_FFT_MIN_TAPS ? 1 : 0;
}
