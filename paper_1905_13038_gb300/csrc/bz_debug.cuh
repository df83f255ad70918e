// Debug build (compiled with -DBZ_DEBUG): every global load and store of the
// window, small-page, stripe, quantile, min/max and Haar kernels is checked
// against the extent of the buffer it belongs to (the image: its H rows of
// pitch bytes; an output: its rows of pitch bytes, the last one only as long
// as the row's data; the library's scratch: its allocation).
// An access outside sets a bit of the translation unit's status word,
// records the first offending address and is skipped (a load then reads 0);
// nothing traps, so the context stays usable and the host reads the status
// (bz_debug_status).  In the normal build the checks compile to nothing.
//
// Status bits: 1 image load, 2 output store, 4 scratch load or store.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime.h>

namespace bz {

constexpr unsigned kDbgImage = 1u, kDbgOutput = 2u, kDbgScratch = 4u;

// Bytes of an image / packed output of `rows` rows: the last row only as far
// as its data reaches.
__host__ __device__ inline size_t dbg_extent(int64_t rows, int64_t pitch, int64_t row_bytes)
{
    return rows < 1 ? 0 : (size_t)((rows - 1) * pitch + row_bytes);
}

#ifdef BZ_DEBUG
// one status per translation unit (no relocatable device code)
static __device__ unsigned int g_dbg_status;
static __device__ unsigned long long g_dbg_addr;

__device__ __forceinline__ bool dbg_in(const void *p, size_t n, const void *base, size_t extent, unsigned code)
{
    const uintptr_t a = (uintptr_t)p, b = (uintptr_t)base;
    if (a >= b && a + n <= b + extent && a + n >= a)
        return true;
    atomicOr(&g_dbg_status, code);
    atomicCAS(&g_dbg_addr, 0ull, (unsigned long long)a);
    return false;
}
#define BZ_DBG_IN(p, n, base, extent, code) ::bz::dbg_in((p), (n), (base), (extent), (code))

// Host accessor of this translation unit's status: copies it out and, with
// reset, clears it.
#define BZ_DEBUG_ACCESSOR(name)                                                                     \
    int name(unsigned *status, unsigned long long *addr, bool reset)                              \
    {                                                                                               \
        unsigned s = 0;                                                                             \
        unsigned long long a = 0;                                                                   \
        if (cudaMemcpyFromSymbol(&s, g_dbg_status, sizeof s) != cudaSuccess ||                     \
            cudaMemcpyFromSymbol(&a, g_dbg_addr, sizeof a) != cudaSuccess)                         \
            return -1;                                                                              \
        *status |= s;                                                                               \
        if (!*addr)                                                                                 \
            *addr = a;                                                                              \
        if (reset) {                                                                                \
            const unsigned z = 0;                                                                   \
            const unsigned long long za = 0;                                                        \
            if (cudaMemcpyToSymbol(g_dbg_status, &z, sizeof z) != cudaSuccess ||                   \
                cudaMemcpyToSymbol(g_dbg_addr, &za, sizeof za) != cudaSuccess)                     \
                return -1;                                                                          \
        }                                                                                           \
        return 0;                                                                                   \
    }
#else
#define BZ_DBG_IN(p, n, base, extent, code) true
#define BZ_DEBUG_ACCESSOR(name)                                                                     \
    int name(unsigned *, unsigned long long *, bool) { return 1; }
#endif

}  // namespace bz
