// Ragged-edge fold kernels of libpcal and the small bookkeeping kernels.
//
// The ragged kernels fold any run of samples at any alignment straight into
// the plan's bins (Eq. 2 with the period L of Eq. 4).  They handle the head
// before the first 16-byte boundary, the tail after the last whole bulk row,
// and inputs too short for the bulk kernel.  2-bit and int8 bins are exact
// integers, so atomic order does not matter; float32 bins are summed by one
// thread per bin in sample order, so they are deterministic.
//
// Every kernel that touches the bins here is launched as a programmatic
// dependent of the kernel before it: it lets its own successor start
// launching at once, then waits for its predecessor (whose adds, or the
// finalize's clearing, come first) before it touches the bins.  The stream's
// kernels therefore still complete in launch order, while their launches
// overlap.
#include "df64.cuh"
#include "internal.cuh"
#include "ptx.cuh"

namespace {

__device__ __forceinline__ void chain_in() {
    pcal_ptx::allow_dependents();
    pcal_ptx::grid_dependency_wait();
}

__global__ void ragged_2bit_kernel(const uint8_t* __restrict__ bytes, int64_t n_bytes, int64_t k0, int64_t L,
                                   unsigned long long* __restrict__ acc) {
    chain_in();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_bytes;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = bytes[i];
        if (b == 0) continue;
        int64_t k = (k0 + 4 * i) % L;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t c = (b >> (2 * j)) & 3u;
            if (c) {
                unsigned long long l = c & 1u, h = c >> 1;
                atomicAdd(&acc[k], l | (h << 21) | ((l & h) << 42));
            }
            if (++k == L) k = 0;
        }
    }
}

__global__ void ragged_i8_kernel(const int8_t* __restrict__ x, int64_t n, int64_t k0, int64_t L,
                                 long long* __restrict__ acc) {
    chain_in();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int v = x[i];
        if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&acc[(k0 + i) % L]), (unsigned long long)(long long)v);
    }
}

// One thread per bin k: sums the samples of this run that fall into bin k, in
// order, in double-float, and adds the sum to the plan's double-float bin.
__global__ void ragged_f32_kernel(const float* __restrict__ x, int64_t n, int64_t k0, int64_t L,
                                  float2* __restrict__ acc) {
    chain_in();
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= L) return;
    int64_t t = (k - k0 % L + L) % L;  // first sample index of this run in bin k
    if (t >= n) return;
    pcal_df::df s{0.f, 0.f};
    for (; t < n; t += L) s = pcal_df::add_f(s, x[t]);
    const float2 a = acc[k];
    s = pcal_df::add(pcal_df::df{a.x, a.y}, s);
    acc[k] = make_float2(s.hi, s.lo);
}

// Move the packed 21-bit fields into the wide 64-bit arrays and clear them.
__global__ void spill2_kernel(unsigned long long* __restrict__ acc, unsigned long long* __restrict__ wide,
                              int64_t L) {
    chain_in();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long v = acc[k];
        if (v) {
            wide[k] += v & PCAL_F21_MASK;
            wide[L + k] += (v >> 21) & PCAL_F21_MASK;
            wide[2 * L + k] += (v >> 42) & PCAL_F21_MASK;
            acc[k] = 0;
        }
    }
}

// Exact per-(bin, code) counts of the current period: [L][4] int64.
__global__ void export2_kernel(const unsigned long long* __restrict__ acc, const unsigned long long* __restrict__ wide,
                               int64_t L, int64_t q, int64_t rem, int64_t a0, long long* __restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long v = acc[k];
        long long sl = (long long)((v & PCAL_F21_MASK) + wide[k]);
        long long sh = (long long)(((v >> 21) & PCAL_F21_MASK) + wide[L + k]);
        long long shl = (long long)(((v >> 42) & PCAL_F21_MASK) + wide[2 * L + k]);
        int64_t r = (k - a0 + L) % L;
        long long cnt = q + (r < rem ? 1 : 0);
        out[4 * k + 3] = shl;
        out[4 * k + 2] = sh - shl;
        out[4 * k + 1] = sl - shl;
        out[4 * k + 0] = cnt - sl - sh + shl;
    }
}

// Failure detection without a fault: every thread of one block waits on an
// mbarrier phase that nothing completes, with the bounded wait of the fold
// kernels and a short limit; each thread that gives up sets a bit, and the
// block then returns normally.
__global__ void wait_timeout_kernel(uint64_t limit_ns, unsigned int* flags) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        pcal_ptx::mbar_init(&bar, (1u << 20) - 1);  // the largest count: more arrivals than will come
        pcal_ptx::fence_barrier_init();
    }
    __syncthreads();
    if (!pcal_ptx::mbar_wait(&bar, 0, limit_ns)) atomicOr(flags, PCAL_DERR_FULL_WAIT);
    __syncthreads();
}

// Launch with programmatic stream serialization (see chain_in).
template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*k)(KArgs...), int grid, int block, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<Args&&>(args)...);
}

inline int grid_for(int64_t work, int threads, int num_sms) {
    int64_t g = (work + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * 8;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

cudaError_t launch_ragged(pcal_plan* p, const uint8_t* d_bytes, int64_t n, int64_t k0, cudaStream_t s) {
    const int64_t L = p->g.L;
    if (n <= 0) return cudaSuccess;
    cudaError_t e;
    switch (p->g.format) {
        case PCAL_2BIT: {
            const int64_t nb = n / 4;
            e = launch_chained(ragged_2bit_kernel, grid_for(nb, 256, p->num_sms), 256, s, d_bytes, nb, k0, L,
                               cur_acc2(p));
            break;
        }
        case PCAL_I8:
            e = launch_chained(ragged_i8_kernel, grid_for(n, 256, p->num_sms), 256, s,
                               reinterpret_cast<const int8_t*>(d_bytes), n, k0, L, cur_acc8(p));
            break;
        default:
            e = launch_chained(ragged_f32_kernel, (int)((L + 255) / 256), 256, s,
                               reinterpret_cast<const float*>(d_bytes), n, k0, L, cur_accf(p));
            break;
    }
    p->stats.kernel_launches += 1;
    return e;
}

cudaError_t launch_spill2(pcal_plan* p, cudaStream_t s) {
    const cudaError_t e =
        launch_chained(spill2_kernel, grid_for(p->g.L, 256, p->num_sms), 256, s, cur_acc2(p), cur_wide2(p), p->g.L);
    p->stats.kernel_launches += 1;
    return e;
}

cudaError_t launch_export_bins(pcal_plan* p, void* d_out, cudaStream_t s) {
    const int64_t L = p->g.L;
    const int64_t n_tot = p->n_abs - p->period_start;
    export2_kernel<<<grid_for(L, 256, p->num_sms), 256, 0, s>>>(cur_acc2(p), cur_wide2(p), L, n_tot / L, n_tot % L,
                                                                  p->period_start % L,
                                                                  reinterpret_cast<long long*>(d_out));
    p->stats.kernel_launches += 1;
    return cudaGetLastError();
}

extern "C" int pcal_selftest_wait_timeout(double limit_s, unsigned int* flags_out) {
    if (!flags_out || !(limit_s > 0.0) || limit_s > 2.0) return PCAL_EINVAL;
    unsigned int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(unsigned int));
    if (e == cudaSuccess) {
        wait_timeout_kernel<<<1, 64>>>((uint64_t)(limit_s * 1e9), d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(flags_out, d, sizeof(unsigned int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return PCAL_ECUDA;
    }
    return *flags_out ? PCAL_ETIMEOUT : PCAL_OK;
}
