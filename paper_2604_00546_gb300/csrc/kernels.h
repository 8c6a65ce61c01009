// Kernel launchers shared by the engine (host-callable, device pointers only).
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>

#include "dev_arith.cuh"

// Programmatic dependent launch. Every kernel of the library starts with pdl_wait(), so it
// touches no memory before the kernel ahead of it in the stream has completed and flushed;
// launched with programmatic stream serialisation, only its launch and CTA scheduling
// overlap the tail of the previous kernel. pdl_trigger() lets the next kernel be scheduled
// once every CTA of this one has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// When launches carry the programmatic-serialisation attribute: FR_PDL=0 never, FR_PDL=1
// always, unset (mode 2) for launches outside stream capture only. Measured on the membership
// match: launched one by one it is about 4% faster with the attribute; replayed as a CUDA graph,
// about 2.5% slower with it.
int pdl_mode();
inline bool pdl_use(cudaStream_t s) {
    const int m = pdl_mode();
    if (m != 2) return m == 1;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusNone;
}

template <typename... KP, typename... A>
inline void launch_k(void (*k)(KP...), dim3 g, dim3 b, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = pdl_use(s) ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, static_cast<KP>(args)...);
}

// cudaFuncSetAttribute acts on the current device only: raise kernel k's dynamic shared memory
// limit once per device (bit d of `done` marks device d). A device is marked only once the
// call has succeeded, so a failed call is retried by the next launch; ordinals 64 and above
// are not cached and set the limit on every launch.
template <class K>
inline void smem_limit_once(K* k, int bytes, std::atomic<unsigned long long>& done) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        return;
    }
    const unsigned long long bit = 1ull << dev;
    if (done.load(std::memory_order_acquire) & bit) return;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess)
        done.fetch_or(bit, std::memory_order_release);
}

#define FR_MAX_PRIMES 64
#define FR_MAX_DIGITS 16

// Periodic prime assignment of a batch of polynomials: poly p uses prime idx[p % period].
struct PrimeMap {
    int period;
    unsigned char idx[FR_MAX_PRIMES];
};

// A batch of N-point polynomials: poly p lives at base + (p / inner) * outer + (p % inner) * N
// and uses prime pm.idx[p % pm.period]. With an index table (tab != nullptr, tab_n entries
// of (offset, prime) pairs) poly p instead lives at base + (p / tab_n) * outer + tab[2e] * N,
// e = p % tab_n, and uses prime tab[2e + 1].
struct PolyBatch {
    u64* base;
    long long outer;
    int inner;
    int npolys;
    PrimeMap pm;
    const int* tab = nullptr;
    int tab_n = 0;
    // optional source of the first pass (out of place): poly p read from
    // src + (p / inner) src_outer + (p % inner) N and written to its place in base
    const u64* src = nullptr;
    long long src_outer = 0;
    // optional second segment (no source, no table): polys split .. npolys - 1 live at
    // base2 + (q / inner2) outer2 + (q % inner2) N, q = p - split, with primes pm2, so the
    // transforms of two buffers share one launch
    int split = 0;
    u64* base2 = nullptr;
    long long outer2 = 0;
    int inner2 = 1;
    PrimeMap pm2{};
};

// NTT batch-size buckets for the tuned tile shapes: <= 4, <= 16, <= 64, larger.
#define FR_NTT_BUCKETS 4
#define FR_NTT_SHAPES 6
__host__ __device__ inline int ntt_bucket(int npolys) {
    return npolys <= 4 ? 0 : npolys <= 16 ? 1 : npolys <= 64 ? 2 : 3;
}

// Ring tables resident on the device for one parameter set.
struct RingDev {
    int logN;
    int N;
    int nprimes;
    const DevPrime* primes;  // [nprimes]
    const ulonglong2* tw;    // [nprimes][N] (psi^brev(k), its Shoup quotient)
    const ulonglong2* itw;   // [nprimes][N] (psi^-brev(k), its Shoup quotient)
    unsigned char ntt_shape[FR_NTT_BUCKETS];  // tile shape per batch-size bucket (see launch_ntt)
};

// Batched negacyclic NTT (evaluation order: position k = value at psi^(2 brev(k)+1)).
void launch_ntt(const RingDev& R, const PolyBatch& b, bool inverse, cudaStream_t s);
// Autotuner of the NTT tile shapes (see ntt.cu); us: FR_NTT_BUCKETS x FR_NTT_SHAPES times in
// microseconds (-1: shape not available), or null.
void tune_ntt(RingDev& R, cudaStream_t s, double* us, int reps);
// Butterflies per second of the NTT's forward butterfly with operands in registers.
double measure_butterfly_peak(int device);
// FP64 operations per second of fused multiply-adds with operands in registers.
double measure_fp64_peak(int device);

// Fast base conversion tables for one (source set, target list).
struct BconvTab {
    int ns;                          // source limbs
    int nt;                          // target limbs
    int src_prime[FR_MAX_DIGITS];    // prime indices of the sources
    int src_pos[FR_MAX_DIGITS];      // positions of the sources in the input layout
    u64 inv_hat[FR_MAX_DIGITS];      // [(B/b_i)^-1]_{b_i}
    u64 inv_hat_s[FR_MAX_DIGITS];
    int tgt_prime[FR_MAX_PRIMES];    // prime index of target t
    int tgt_pos[FR_MAX_PRIMES];      // position of target t in the output layout
};
// hat[i][t] = [B/b_i]_{q_t}, with Shoup quotients; stored on the device as [ns][nt] pairs
