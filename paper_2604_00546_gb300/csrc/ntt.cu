// Batched negacyclic NTT / inverse NTT over 64-bit primes.
//
// Forward: Cooley-Tukey with twiddles psi^brev(k) (natural-order input,
// evaluation order output: position k = A(psi^(2 brev(k)+1))). Inverse:
// Gentleman-Sande with psi^-brev(k), then N^-1. The log N stages are split
// in two shared-memory passes over an R x C view of the polynomial
// (N = R * C): the first log R stages only couple elements of one column
// (stride C), the remaining log C stages only couple elements of one row
// (contiguous). Each pass loads a tile to shared memory once, runs its stages
// there and writes back once, so a transform costs two streaming passes; for
// a batch of limbs that fits in L2 the intermediate stays on chip.
#include "kernels.h"

namespace {

constexpr int kTC = 16;  // columns per tile in the column pass

__device__ __forceinline__ u64* poly_ptr(const PolyBatch& b, int p, int N) {
    return b.base + (long long)(p / b.inner) * b.outer + (long long)(p % b.inner) * N;
}

template <bool INV>
__global__ void __launch_bounds__(256) k_ntt_col(RingDev R, PolyBatch b, int logR) {
    extern __shared__ u64 sm[];
    const int N = R.N;
    const int Rr = 1 << logR;
    const int C = N >> logR;
    const int p = blockIdx.y;
    u64* x = poly_ptr(b, p, N);
    const int pi = b.pm.idx[p % b.pm.period];
    const DevPrime P = R.primes[pi];
    const u64 q = P.q;
    const u64* tw = (INV ? R.itw : R.tw) + (size_t)pi * N;
    const u64* tws = (INV ? R.itws : R.tws) + (size_t)pi * N;
    u64* s = sm;
    u64* sw = sm + Rr * kTC;
    u64* sws = sw + Rr;
    const int col0 = blockIdx.x * kTC;
    for (int i = threadIdx.x; i < Rr; i += blockDim.x) {
        sw[i] = tw[i];
        sws[i] = tws[i];
    }
    for (int e = threadIdx.x; e < Rr * kTC; e += blockDim.x) {
        int r = e / kTC, c = e - r * kTC;
        s[e] = x[(long long)r * C + col0 + c];
    }
    __syncthreads();
    const int half = (Rr >> 1) * kTC;
    if (!INV) {
        for (int m = 1, h = Rr >> 1; m < Rr; m <<= 1, h >>= 1) {
            for (int bf = threadIdx.x; bf < half; bf += blockDim.x) {
                int c = bf % kTC, pr = bf / kTC;
                int i = pr / h, u = pr - i * h;
                int ra = i * 2 * h + u, rb = ra + h;
                u64 U = s[ra * kTC + c];
                u64 V = mul_shoup(s[rb * kTC + c], sw[m + i], sws[m + i], q);
                s[ra * kTC + c] = add_mod(U, V, q);
                s[rb * kTC + c] = sub_mod(U, V, q);
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < Rr * kTC; e += blockDim.x) {
            int r = e / kTC, c = e - r * kTC;
            x[(long long)r * C + col0 + c] = s[e];
        }
    } else {
        for (int m = Rr >> 1, h = 1; m >= 1; m >>= 1, h <<= 1) {
            for (int bf = threadIdx.x; bf < half; bf += blockDim.x) {
                int c = bf % kTC, pr = bf / kTC;
                int i = pr / h, u = pr - i * h;
                int ra = i * 2 * h + u, rb = ra + h;
                u64 U = s[ra * kTC + c];
                u64 V = s[rb * kTC + c];
                s[ra * kTC + c] = add_mod(U, V, q);
                s[rb * kTC + c] = mul_shoup(sub_mod(U, V, q), sw[m + i], sws[m + i], q);
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < Rr * kTC; e += blockDim.x) {
            int r = e / kTC, c = e - r * kTC;
            x[(long long)r * C + col0 + c] = mul_shoup(s[e], P.ninv, P.ninv_s, q);
        }
    }
}

template <bool INV>
__global__ void __launch_bounds__(256) k_ntt_row(RingDev R, PolyBatch b, int logR, int bpc) {
    extern __shared__ u64 sm[];
    const int N = R.N;
    const int C = N >> logR;
    const int p = blockIdx.y;
    u64* x = poly_ptr(b, p, N);
    const int pi = b.pm.idx[p % b.pm.period];
    const u64 q = R.primes[pi].q;
    const u64* tw = (INV ? R.itw : R.tw) + (size_t)pi * N;
    const u64* tws = (INV ? R.itws : R.tws) + (size_t)pi * N;
    const int tile = bpc * C;
    const long long g0 = (long long)blockIdx.x * tile;
    for (int e = threadIdx.x; e < tile; e += blockDim.x) sm[e] = x[g0 + e];
    __syncthreads();
    const int hc = C >> 1;
    const int half = tile >> 1;
    if (!INV) {
        long long m = 1ll << logR;
        for (int t = hc; t >= 1; t >>= 1, m <<= 1) {
            for (int bf = threadIdx.x; bf < half; bf += blockDim.x) {
                int blk = bf / hc, pp = bf - blk * hc;
                int il = pp / t, u = pp - il * t;
                int ja = blk * C + il * 2 * t + u, jb = ja + t;
                long long widx = m + (g0 + ja) / (2 * t);
                u64 U = sm[ja];
                u64 V = mul_shoup(sm[jb], __ldg(tw + widx), __ldg(tws + widx), q);
                sm[ja] = add_mod(U, V, q);
                sm[jb] = sub_mod(U, V, q);
            }
            __syncthreads();
        }
    } else {
        long long m = (long long)N >> 1;
        for (int t = 1; t <= hc; t <<= 1, m >>= 1) {
            for (int bf = threadIdx.x; bf < half; bf += blockDim.x) {
                int blk = bf / hc, pp = bf - blk * hc;
                int il = pp / t, u = pp - il * t;
                int ja = blk * C + il * 2 * t + u, jb = ja + t;
                long long widx = m + (g0 + ja) / (2 * t);
                u64 U = sm[ja];
                u64 V = sm[jb];
                sm[ja] = add_mod(U, V, q);
                sm[jb] = mul_shoup(sub_mod(U, V, q), __ldg(tw + widx), __ldg(tws + widx), q);
            }
            __syncthreads();
        }
    }
    for (int e = threadIdx.x; e < tile; e += blockDim.x) x[g0 + e] = sm[e];
}

}  // namespace

void launch_ntt(const RingDev& R, const PolyBatch& b, bool inverse, cudaStream_t s) {
    if (b.npolys <= 0) return;
    const int logN = R.logN;
    const int logR = logN / 2;
    const int Rr = 1 << logR;
    const int C = R.N >> logR;
    int bpc = 2048 / C;
    if (bpc < 1) bpc = 1;
    if (bpc > Rr) bpc = Rr;
    const size_t smc = (size_t)(Rr * kTC + 2 * Rr) * sizeof(u64);
    const size_t smr = (size_t)bpc * C * sizeof(u64);
    dim3 gc(C / kTC, b.npolys), gr(Rr / bpc, b.npolys);
    if (!inverse) {
        k_ntt_col<false><<<gc, 256, smc, s>>>(R, b, logR);
        k_ntt_row<false><<<gr, 256, smr, s>>>(R, b, logR, bpc);
    } else {
        k_ntt_row<true><<<gr, 256, smr, s>>>(R, b, logR, bpc);
        k_ntt_col<true><<<gc, 256, smc, s>>>(R, b, logR);
    }
}
