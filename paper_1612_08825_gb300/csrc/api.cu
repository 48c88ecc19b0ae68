// Status strings, version and CUDA-error bookkeeping of the fastttc C ABI.
#include <atomic>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tma.cuh"

namespace ft {

static thread_local char g_cuda_error[256] = "";

void set_cuda_error(cudaError_t e)
{
    const char *s = cudaGetErrorString(e);
    std::strncpy(g_cuda_error, s ? s : "unknown CUDA error", sizeof(g_cuda_error) - 1);
    g_cuda_error[sizeof(g_cuda_error) - 1] = '\0';
}

static std::atomic<unsigned> g_tma_extra_tx{0};

unsigned tma_extra_tx() { return g_tma_extra_tx.load(); }

void set_tma_extra_tx(unsigned v) { g_tma_extra_tx.store(v); }

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        cudaGetLastError();
    });
    return fn;
}

}  // namespace ft

extern "C" const char *ft_status_string(int status)
{
    switch (status) {
    case FT_OK: return "FT_OK";
    case FT_ERR_INVALID_ARG: return "FT_ERR_INVALID_ARG";
    case FT_ERR_SHAPE: return "FT_ERR_SHAPE";
    case FT_ERR_UNSUPPORTED: return "FT_ERR_UNSUPPORTED";
    case FT_ERR_WORKSPACE: return "FT_ERR_WORKSPACE";
    case FT_ERR_CUDA: return "FT_ERR_CUDA";
    case FT_ERR_TIMEOUT: return "FT_ERR_TIMEOUT";
    default: return "FT_ERR_UNKNOWN";
    }
}

extern "C" const char *ft_last_cuda_error(void) { return ft::g_cuda_error; }

extern "C" int ft_version(void) { return 1 * 10000 + 0 * 100 + 0; }

extern "C" void ft_test_stall_tma_waits(int on) { ft::set_tma_extra_tx(on ? 16u : 0u); }
