// cher_pack.cu -- the records of every telescope packed contiguously,
// telescope after telescope, for one download instead of one per telescope.
// Every CTA scans the (clipped) counts into shared memory; threads then
// stride over the packed records, each finding its telescope by a binary
// search over those offsets, with coalesced reads and writes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "cher_internal.h"

namespace cher {
namespace {

struct alignas(16) D4 {
    double2 a, b;
};

template <class V>
__global__ void __launch_bounds__(256) k_pack(const V *pos, const V *tim, const uint64_t *key,
                                              const unsigned long long *count, int64_t cap,
                                              int n_tel, int64_t max_rec, V *dpos, V *dtim,
                                              uint64_t *dkey, int64_t *off) {
    extern __shared__ int64_t s_off[];   // n_tel + 1
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int k = 0; k < n_tel; ++k) {
            s_off[k] = acc;
            const unsigned long long c = count[k];
            acc += static_cast<int64_t>(c < static_cast<unsigned long long>(cap) ? c : cap);
        }
        s_off[n_tel] = acc;
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int k = threadIdx.x; k <= n_tel; k += blockDim.x) off[k] = s_off[k];
    const int64_t total = s_off[n_tel] < max_rec ? s_off[n_tel] : max_rec;
    for (int64_t d = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; d < total;
         d += int64_t(gridDim.x) * blockDim.x) {
        int lo = 0, hi = n_tel;              // the last k with s_off[k] <= d
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_off[mid] <= d) lo = mid; else hi = mid;
        }
        const int64_t src = static_cast<int64_t>(lo) * cap + (d - s_off[lo]);
        dpos[d] = pos[src];
        dtim[d] = tim[src];
        dkey[d] = key[src];
    }
}

}  // namespace

cudaError_t pack_records(bool fp32, const void *pos, const void *tim, const uint64_t *key,
                         const unsigned long long *count, int64_t cap, int n_tel, int64_t max_rec,
                         void *dpos, void *dtim, uint64_t *dkey, int64_t *off, int num_sms,
                         void *stream) {
    const size_t smem = sizeof(int64_t) * (static_cast<size_t>(n_tel) + 1);
    const int grid = std::max(1, num_sms * 4);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (fp32)
        k_pack<float4><<<grid, 256, smem, st>>>(
            static_cast<const float4 *>(pos), static_cast<const float4 *>(tim), key, count, cap,
            n_tel, max_rec, static_cast<float4 *>(dpos), static_cast<float4 *>(dtim), dkey, off);
    else
        k_pack<D4><<<grid, 256, smem, st>>>(
            static_cast<const D4 *>(pos), static_cast<const D4 *>(tim), key, count, cap, n_tel,
            max_rec, static_cast<D4 *>(dpos), static_cast<D4 *>(dtim), dkey, off);
    return cudaGetLastError();
}

}  // namespace cher
