// rebk_device.cuh -- device helpers shared by the REBK kernels (sm_103a).
//
// * Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11),
//   written from that paper: key (seed, stream), counter (d, 0, 0, 0).
// * Block pick of Algorithm 1 (Du, Si, Sun, arXiv:2001.04179): the smallest
//   block index whose cumulative squared Frobenius norm exceeds u ||A||_F^2.
// * 16-byte vector loads of FP64 / FP32 / BF16 storage.
// * A device-wide barrier for the persistent kernel: release/acquire on a
//   monotonic counter, with a wall-clock limit so that no wait is unbounded.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rebk {

// ---------------------------------------------------------------------------
// Philox4x64-10
// ---------------------------------------------------------------------------
struct PhiloxOut {
    uint64_t w[4];
};

__device__ __forceinline__ PhiloxOut philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                                   uint64_t c3, uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
        const uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
        const uint64_t n0 = hi1 ^ c1 ^ k0;
        const uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    PhiloxOut o;
    o.w[0] = c0; o.w[1] = c1; o.w[2] = c2; o.w[3] = c3;
    return o;
}

// u in [0, 1) for draw d of stream (seed, stream).
__device__ __forceinline__ double draw_uniform(uint64_t seed, uint64_t stream, uint64_t d) {
    const PhiloxOut o = philox4x64_10(d, 0, 0, 0, seed, stream);
    return (double)(o.w[0] >> 11) * 0x1.0p-53;
}

// u in [0, 1) for slot q of draw d: counter (d, q, 0, 0); slot 0 is draw_uniform.
__device__ __forceinline__ double draw_uniform_slot(uint64_t seed, uint64_t stream, uint64_t d, uint64_t q) {
    const PhiloxOut o = philox4x64_10(d, q, 0, 0, seed, stream);
    return (double)(o.w[0] >> 11) * 0x1.0p-53;
}

// Smallest b in [0, nb) with cdf[b] > u * cdf[nb-1]; if none (the product
// rounded to the total), the fallback block (last one of nonzero norm).
__device__ __forceinline__ int pick_block(const double *cdf, int nb, double u, int fallback) {
    const double target = __dmul_rn(u, cdf[nb - 1]);
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cdf[mid] > target) hi = mid;
        else lo = mid + 1;
    }
    return cdf[lo] > target ? lo : fallback;
}

// ---------------------------------------------------------------------------
// 16-byte vector loads, converted to the arithmetic type
// ---------------------------------------------------------------------------
template <typename TA, typename TS> struct VecIO;

template <> struct VecIO<double, double> {
    static constexpr int V = 2;
    __device__ __forceinline__ static void load(const double *p, double (&o)[2]) {
        const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
        o[0] = v.x; o[1] = v.y;
    }
    __device__ __forceinline__ static void load_generic(const double *p, double (&o)[2]) {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        o[0] = v.x; o[1] = v.y;
    }
    __device__ __forceinline__ static void load_shared(uint32_t a, double (&o)[2]) {
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(o[0]), "=d"(o[1]) : "r"(a));
    }
    // the V arithmetic-type values that pair with one stored vector
    __device__ __forceinline__ static void load_shared_ts(uint32_t a, double (&o)[2]) { load_shared(a, o); }
    __device__ __forceinline__ static void zero(double (&o)[2]) { o[0] = o[1] = 0.0; }
};

template <> struct VecIO<float, float> {
    static constexpr int V = 4;
    __device__ __forceinline__ static void load(const float *p, float (&o)[4]) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    __device__ __forceinline__ static void load_generic(const float *p, float (&o)[4]) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    __device__ __forceinline__ static void load_shared(uint32_t a, float (&o)[4]) {
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]) : "r"(a));
    }
    __device__ __forceinline__ static void load_shared_ts(uint32_t a, float (&o)[4]) { load_shared(a, o); }
    __device__ __forceinline__ static void zero(float (&o)[4]) { o[0] = o[1] = o[2] = o[3] = 0.f; }
};

template <> struct VecIO<__nv_bfloat16, float> {
    static constexpr int V = 8;
    __device__ __forceinline__ static void unpack(const uint4 v, float (&o)[8]) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            o[2 * i] = __uint_as_float(w[i] << 16);
            o[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
        }
    }
    __device__ __forceinline__ static void load(const __nv_bfloat16 *p, float (&o)[8]) {
        unpack(__ldg(reinterpret_cast<const uint4 *>(p)), o);
    }
    __device__ __forceinline__ static void load_generic(const __nv_bfloat16 *p, float (&o)[8]) {
        unpack(*reinterpret_cast<const uint4 *>(p), o);
    }
    __device__ __forceinline__ static void load_shared(uint32_t a, float (&o)[8]) {
        uint4 v;
        asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
        unpack(v, o);
    }
    __device__ __forceinline__ static void load_shared_ts(uint32_t a, float (&o)[8]) {
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]) : "r"(a));
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(o[4]), "=f"(o[5]), "=f"(o[6]), "=f"(o[7]) : "r"(a + 16u));
    }
    __device__ __forceinline__ static void zero(float (&o)[8]) {
#pragma unroll
        for (int i = 0; i < 8; ++i) o[i] = 0.f;
    }
};

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Loads that bypass L1: data written by other CTAs during this launch.
__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ double ld_cg_t(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg_t(const float *p) { return __ldcg(p); }

// ---------------------------------------------------------------------------
// L2 prefetch of a byte range (rounded out to 16-byte boundaries)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void prefetch_l2_range(const void *begin, const void *end) {
    uintptr_t a = reinterpret_cast<uintptr_t>(begin) & ~uintptr_t(15);
    uintptr_t b = (reinterpret_cast<uintptr_t>(end) + 15) & ~uintptr_t(15);
    if (b <= a) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(b - a))
                 : "memory");
}

// ---------------------------------------------------------------------------
// Device-wide barrier with a wall-clock limit
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_gpu_add(unsigned int *p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Split-phase device barrier.  grid_arrive: after the CTA's writes of a
// phase (all threads call it; thread 0 releases them at gpu scope).
__device__ __forceinline__ void grid_arrive(unsigned int *counter) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        red_release_gpu_add(counter, 1u);
    }
}

// grid_wait: until *counter >= target (all threads call it); false for every
// thread of the CTA if the wait ran past timeout_ns (status set to TIMEOUT).
__device__ __forceinline__ bool grid_wait(unsigned int *counter, unsigned int target, int *status,
                                          unsigned long long timeout_ns, int *s_flag) {
    if (threadIdx.x == 0) {
        int ok = 1;
        if (ld_acquire_gpu(counter) < target) {
            const unsigned long long t0 = globaltimer_ns();
            unsigned int spins = 0;
            while (ld_acquire_gpu(counter) < target) {
                if ((++spins & 255u) == 0u && globaltimer_ns() - t0 > timeout_ns) {
                    ok = 0;
                    atomicExch(status, 6 /* REBK_BARRIER_TIMEOUT */);
                    break;
                }
            }
        }
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// All CTAs of the launch call this with the same target = gridDim.x * (phase + 1).
// Returns false (for every thread of the CTA) if the wait ran past timeout_ns;
// the CTA then records the timeout in *status and must leave the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned int *counter, unsigned int target,
                                             int *status, unsigned long long timeout_ns,
                                             int *s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        red_release_gpu_add(counter, 1u);
        int ok = 1;
        if (ld_acquire_gpu(counter) < target) {
            const unsigned long long t0 = globaltimer_ns();
            unsigned int spins = 0;
            while (ld_acquire_gpu(counter) < target) {
                if ((++spins & 255u) == 0u && globaltimer_ns() - t0 > timeout_ns) {
                    ok = 0;
                    atomicExch(status, 6 /* REBK_BARRIER_TIMEOUT */);
                    break;
                }
            }
        }
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

}  // namespace rebk
