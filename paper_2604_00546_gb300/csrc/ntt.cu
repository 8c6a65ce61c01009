// Batched negacyclic NTT / inverse NTT over 64-bit primes.
//
// Forward: Cooley-Tukey with twiddles psi^brev(k) (natural-order input,
// evaluation-order output: position k = A(psi^(2 brev(k)+1))). Inverse:
// Gentleman-Sande with psi^-brev(k), then N^-1.
//
// The log N stages are split in two passes over an R x C view of the
// polynomial (N = R C): the first log R stages only couple elements of one
// column (stride C), the remaining log C stages only couple elements of one
// row (contiguous). Each pass loads its tile once and writes it once. Inside a
// pass every thread keeps 8 elements in registers and runs up to 3 radix-2
// stages on them; the elements are re-distributed through shared memory
// between these 3-stage phases, so a 256-point sub-transform costs 2
// exchanges instead of 8. Index arithmetic is shifts and masks only.
//
// Residues stay lazily reduced (Harvey): forward butterflies keep values in
// [0, 4q), inverse butterflies in [0, 2q); the last pass returns [0, q).
// Twiddle of the butterfly pairing x and x + 2^b, in either direction:
// tw[(M + J) >> (b + 1)] where J is the global index of x and M = R for the
// column pass, N for the row pass.
#include <cooperative_groups.h>
#include <cstdlib>
#include <type_traits>

#include "ckks_kernels.h"

namespace {


__device__ __forceinline__ u64* poly_at(const PolyBatch& b, int p, int N, int* prime) {
    if (b.split && p >= b.split) {
        const int q = p - b.split;
        *prime = b.pm2.idx[q % b.pm2.period];
        return b.base2 + (long long)(q / b.inner2) * b.outer2 + (long long)(q % b.inner2) * N;
    }
    if (b.tab) {
        const int e = p % b.tab_n;
        *prime = __ldg(b.tab + 2 * e + 1);
        return b.base + (long long)(p / b.tab_n) * b.outer + (long long)__ldg(b.tab + 2 * e) * N;
    }
    *prime = b.pm.idx[p % b.pm.period];
    return b.base + (long long)(p / b.inner) * b.outer + (long long)(p % b.inner) * N;
}

// where the first pass reads poly p: its source when the batch has one, else its place
__device__ __forceinline__ const u64* poly_in(const PolyBatch& b, int p, int N, const u64* x) {
    return b.src ? b.src + (long long)(p / b.inner) * b.src_outer + (long long)(p % b.inner) * N : x;
}

__device__ __forceinline__ u64 shoup_lazy(u64 x, u64 w, u64 ws, u64 q) {
    return x * w - __umul64hi(x, ws) * q;  // in [0, 2q)
}

// element index of register e of thread tau in a phase whose 3 bits start at LO
template <int LO>
__device__ __forceinline__ int phase_x(int tau, int e) {
    return ((tau >> LO) << (LO + 3)) | (e << LO) | (tau & ((1 << LO) - 1));
}

template <int LOG, bool INV, int PH>
struct PhaseInfo {
    // forward phases take bits in descending order, inverse ones ascending;
    // a phase covers the 3 bits [LO, LO + 3) and runs the stages on bits [BFROM, BTO)
    static constexpr int LO = INV ? (3 * PH < LOG - 3 ? 3 * PH : LOG - 3) : (LOG - 3 * (PH + 1) > 0 ? LOG - 3 * (PH + 1) : 0);
    static constexpr int BFROM = INV ? 3 * PH : LO;
    static constexpr int BTO = INV ? (3 * PH + 3 < LOG ? 3 * PH + 3 : LOG) : LOG - 3 * PH;
};

// Twiddles of a pass: (w, Shoup quotient) pairs, one 16-byte load each. GLOBAL: the table
// itself (read-only path), else a copy staged in shared memory.
template <bool GLOBAL>
struct Ctx {
    int Jbase, M;    // global index of the tile's element 0; M = R (column pass) or N (row pass)
    const ulonglong2* tw;
    u64 q;
    bool grow;       // forward only: q < 2^57, values may grow by 2q per stage (16 stages < 33q < 2^62)
    __device__ __forceinline__ ulonglong2 ld(int i) const {
        if constexpr (GLOBAL) return __ldg(tw + i);
        else return tw[i];
    }
};

// One radix-2 stage on bit B of the registers of a phase with base bit LO. The butterfly of
// registers e and e + 2^lb (lb = B - LO) takes twiddle (M + J + x) >> (B + 1), x its element
// index: M + J and the thread's bits of x above LO + 3 are multiples of 2^(B+1), and x's bits
// below B + 1 are e's bits up to lb and the thread's bits below LO, so the twiddle is
// base + (e >> (lb + 1)): the stage needs 4 >> lb distinct twiddles, loaded before its
// butterflies run.
template <bool INV, int LO, int B, class C>
__device__ __forceinline__ void stage(u64 (&v)[8], int tau, const C& c) {
    constexpr int lb = B - LO;
    constexpr int NT = 4 >> lb;
    const u64 q2 = 2 * c.q;
    const int base = (c.M + c.Jbase + ((tau >> LO) << (LO + 3))) >> (B + 1);
    ulonglong2 w[NT];
#pragma unroll
    for (int u = 0; u < NT; ++u) w[u] = c.ld(base + u);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        if (e & (1 << lb)) continue;
        const int e1 = e | (1 << lb);
        const ulonglong2 t = w[e >> (lb + 1)];
        if (!INV) {
            u64 X = v[e];
            if (!c.grow) X = X >= q2 ? X - q2 : X;
            const u64 T = shoup_lazy(v[e1], t.x, t.y, c.q);
            v[e] = X + T;
            v[e1] = X - T + q2;
        } else {
            const u64 X = v[e], Y = v[e1];
            u64 S = X + Y;
            S = S >= q2 ? S - q2 : S;
            v[e] = S;
            v[e1] = shoup_lazy(X - Y + q2, t.x, t.y, c.q);
        }
    }
}

template <bool INV, int LO, int BFROM, int BTO, int K, class C>
__device__ __forceinline__ void stages(u64 (&v)[8], int tau, const C& c) {
    // forward: bits BTO-1 down to BFROM; inverse: BFROM up to BTO-1
    if constexpr (K < BTO - BFROM) {
        constexpr int B = INV ? BFROM + K : BTO - 1 - K;
        stage<INV, LO, B>(v, tau, c);
        stages<INV, LO, BFROM, BTO, K + 1>(v, tau, c);
    }
}

template <int LOG, bool INV, int PH, class Ex, class C>
__device__ __forceinline__ void phases(u64 (&v)[8], int tau, const C& c, Ex& ex) {
    constexpr int P = (LOG + 2) / 3;
    if constexpr (PH < P) {
        using I = PhaseInfo<LOG, INV, PH>;
        if constexpr (PH > 0) {
            using Prev = PhaseInfo<LOG, INV, PH - 1>;
            ex.template exchange<Prev::LO, I::LO>(v, tau);
        }
        stages<INV, I::LO, I::BFROM, I::BTO, 0>(v, tau, c);
        phases<LOG, INV, PH + 1>(v, tau, c, ex);
    }
}

template <int LOG, bool INV>
struct LastLo {
    static constexpr int v = PhaseInfo<LOG, INV, (LOG + 2) / 3 - 1>::LO;
};

__device__ __forceinline__ u64 reduce4(u64 x, u64 q) {
    x = x >= 2 * q ? x - 2 * q : x;
    return x >= q ? x - q : x;
}

// exchange through shared memory, column layout s[x'][KTC]. With 4 columns x' = x ^ x3 ^
// (x4 << 1), with 8 columns x' = x ^ x3: the rows a half-warp touches then fall on distinct
// bank groups in every phase layout.
template <int KTC>
__device__ __forceinline__ int col_row(int x) {
    return KTC == 4 ? x ^ ((x >> 3) & 1) ^ (((x >> 4) & 1) << 1) : x ^ ((x >> 3) & 1);
}

template <int KTC>
struct ColEx {
    u64* s;
    int col;
    template <int LA, int LB>
    __device__ __forceinline__ void exchange(u64 (&v)[8], int tau) {
#pragma unroll
        for (int e = 0; e < 8; ++e) s[col_row<KTC>(phase_x<LA>(tau, e)) * KTC + col] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = s[col_row<KTC>(phase_x<LB>(tau, e)) * KTC + col];
        __syncthreads();
    }
};

// Shared-memory word of element x of a row: the low 4 bits are XORed with bits 4..6
// (x4 -> bit 0, x5 -> bit 2, x6 -> bits 1 and 3). For 256-point rows this keeps every
// half-warp access of the forward (bits from 5, 2, 0) and inverse (0, 3, 5) phase layouts
// on 16 distinct 8-byte bank pairs.
__device__ __forceinline__ int row_swz(int x) {
    return x ^ ((x >> 4) & 1) ^ (((x >> 5) & 1) << 2) ^ (((x >> 6) & 1) * 10);
}

// exchange through shared memory, one row
struct RowEx {
    u64* s;
    template <int LA, int LB>
    __device__ __forceinline__ void exchange(u64 (&v)[8], int tau) {
#pragma unroll
        for (int e = 0; e < 8; ++e) s[row_swz(phase_x<LA>(tau, e))] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = s[row_swz(phase_x<LB>(tau, e))];
        __syncthreads();
    }
};

// column pass: one CTA = KTC columns x S rows; thread (tau, col) with col = threadIdx % KTC
template <int LOG, bool INV, int KTC>
__global__ void __launch_bounds__(KTC * (1 << LOG) / 8, 5) k_ntt_col(const __grid_constant__ RingDev R, const __grid_constant__ PolyBatch b) {
    pdl_wait();
    pdl_trigger();
    constexpr int S = 1 << LOG;
    extern __shared__ u64 sm[];
    ulonglong2* sw = reinterpret_cast<ulonglong2*>(sm + S * KTC);  // twiddles [0, S)
    const int N = R.N;
    const int C = N >> LOG;
    const int p = blockIdx.y;
    int pi;
    u64* x = poly_at(b, p, N, &pi);
    const u64 q = R.primes[pi].q;
    const ulonglong2* tw = (INV ? R.itw : R.tw) + (size_t)pi * N;
    for (int i = threadIdx.x; i < S; i += blockDim.x) sw[i] = __ldg(tw + i);
    const int col = threadIdx.x & (KTC - 1);
    const int tau = threadIdx.x / KTC;
    const int gcol = blockIdx.x * KTC + col;
    constexpr int L0 = PhaseInfo<LOG, INV, 0>::LO;
    constexpr int LL = LastLo<LOG, INV>::v;
    const u64* xin = INV ? x : poly_in(b, p, N, x);  // the column pass is the forward transform's first
    u64 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = xin[(long long)phase_x<L0>(tau, e) * C + gcol];
    __syncthreads();
    Ctx<false> c{0, S, sw, q, q < (1ull << 57)};
    ColEx<KTC> ex{sm, col};
    phases<LOG, INV, 0>(v, tau, c, ex);
    if (INV) {
        const DevPrime P = R.primes[pi];
#pragma unroll
        for (int e = 0; e < 8; ++e)
            x[(long long)phase_x<LL>(tau, e) * C + gcol] = mul_shoup(v[e], P.ninv, P.ninv_s, q);
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) x[(long long)phase_x<LL>(tau, e) * C + gcol] = v[e];
    }
}

// Epilogues of the forward row pass (the last pass of a forward transform): instead of
// storing the transformed value v (canonical) of poly p at index k in place, the fused
// epilogue finishes the operation the transform belonged to.
struct EpiStore {};

// Montgomery form of the transformed value, stored in place (template diagonals).
struct EpiToMont {};

// ModDown combine: poly p = (job, component t, limb i) of the P -> Q conversions; out =
// (acc_Q - v) P^-1 (+ sigma_g(c0) for rotations, + the ct addend for relinearisation; a
// rotation may add a ciphertext as well, as in x + Rot(x)).
struct EpiModDown {
    MDJobs jobs;
    int npos, level, logN;
    const u64* pinv;
    const u64* pinv_s;
    __device__ __forceinline__ void put(int p, int k, u64 v, u64 q) const {
        const int L1 = level + 1, N = 1 << logN;
        const int j = p / (2 * L1), r = p % (2 * L1), t = r / L1, i = r % L1;
        const MDJob& J = jobs.j[j];
        const u64 a = J.acc[((long long)t * npos + i) * N + k];
        u64 w = mul_shoup(sub_mod(a, v, q), pinv[i], pinv_s[i], q);
        if (J.mode == 1 || J.mode == 3) {
            if (t == 0) w = add_mod(w, J.add[(long long)i * N + galois_src_index((u32)k, J.galois, logN)], q);
            if (J.mode == 3) w = add_mod(w, J.add2[((long long)t * J.add_cap + i) * N + k], q);
        } else if (J.mode == 2) {
            w = add_mod(w, J.add[((long long)t * J.add_cap + i) * N + k], q);
        }
        J.out[((long long)t * J.out_cap + i) * N + k] = w;
    }
};

// Rescale combine: poly p = (ct component bt, limb i) of the lifted last limb;
// out = (x - v) q_l^-1, then (mode 1) + the matching component of an addend ct, or
// (mode 2) doubled with cres_i subtracted from component 0 (2 T^2 - 1 of the Chebyshev powers).
struct EpiRescale {
    const u64* x;
    u64* out;
    const RescaleTab* tab;
    int x_cap, out_cap, l, N;
    int mode;
    const u64* add;     // mode 1: ct b at add + b add_bs, component t at + t add_cap N
    int add_cap;
    long long add_bs;
    const u64* cres;    // mode 2: [l] constants
    __device__ __forceinline__ void put(int p, int k, u64 v, u64 q) const {
        const int bt = p / l, i = p % l;
        const u64 a = x[((long long)bt * x_cap + i) * N + k];
        u64 r = mul_shoup(sub_mod(a, v, q), tab->qlinv[i], tab->qlinv_s[i], q);
        if (mode == 1) {
            r = add_mod(r, add[(long long)(bt >> 1) * add_bs + ((long long)(bt & 1) * add_cap + i) * N + k], q);
        } else if (mode == 2) {
            r = add_mod(r, r, q);
            if ((bt & 1) == 0) r = sub_mod(r, cres[i], q);
        }
        out[((long long)bt * out_cap + i) * N + k] = r;
    }
};

// Rescale of the Chebyshev leaves Rescale(T1 cb_j + ca_j) without the leaves in memory: poly
// p = ((b nl + j) 2 + t) l + i of the lifted last limbs; the leaf's limb i,
// x_i cb_{j,i} (+ ca_{j,i} on component 0), is formed from T1 (query b at x + b x_bs) with the
// same operations as the leaf kernel that stores it, then out = (leaf_i - v) q_l^-1, leaf (b, j)
// at out + (b nl + j) 2 out_cap N. Bit for bit the leaves stored, then rescaled.
struct EpiLeafRescale {
    const u64* x;
    long long x_bs;
    int x_cap;
    const u64* cb;      // [nl][L1] residues of round(c1 Delta)
    const u64* cb_s;    // their Shoup quotients
    const u64* ca;      // [nl][L1] residues of round(c0 Delta) Delta
    int nl, L1;
    u64* out;
    int out_cap;
    const RescaleTab* tab;
    int l, N;
    __device__ __forceinline__ void put(int p, int k, u64 v, u64 q) const {
        const int bjt = p / l, i = p % l, t = bjt & 1, bj = bjt >> 1, j = bj % nl, b = bj / nl;
        u64 a = mul_shoup(x[(long long)b * x_bs + ((long long)t * x_cap + i) * N + k], cb[j * L1 + i], cb_s[j * L1 + i], q);
        if (t == 0) a = add_mod(a, ca[j * L1 + i], q);
        out[((long long)bjt * out_cap + i) * N + k] = mul_shoup(sub_mod(a, v, q), tab->qlinv[i], tab->qlinv_s[i], q);
    }
};

// Relinearisation ModDown fused with the rescale after it (the product of two ciphertexts at
// level l, relinearised, then divided by q_l): poly p = (job j, component t, limb i < l) of
// y = conv P^-1 + lift, where conv is the ModDown's P -> Q conversion and lift the centered last
// limb of the ModDown's output. out = (acc_i P^-1 + d_i - v) q_l^-1 with acc the job's key-switch
// inner product [2][npos][N] and d its tensor product [3][l+1][N] (d0, d1 the addend; null: no
// addend, a plain ModDown then rescale); then the modes of EpiRescale. Each step is exact modular arithmetic and the NTT is linear, so this equals
// ModDown, the addition of (d0, d1) and the rescale one after the other, bit for bit.
struct EpiRelinRescale {
    const u64* acc;
    const u64* d;
    u64* out;          // job j at out + j out_bs, component t at + t out_cap N
    const RescaleTab* tab;
    const u64* pinv;
    const u64* pinv_s;
    int npos, l, N, out_cap, mode;
    long long out_bs;
    const u64* add;    // mode 1: job j's addend at add + j add_bs, component t at + t add_cap N
    int add_cap;
    long long add_bs;
    const u64* cres;   // mode 2: [l] constants
    __device__ __forceinline__ void put(int p, int k, u64 v, u64 q) const {
        const int jt = p / l, i = p % l, j = jt >> 1, t = jt & 1;
        const u64 a = acc[((long long)jt * npos + i) * N + k];
        const u64 dd = d ? d[(((long long)j * 3 + t) * (l + 1) + i) * N + k] : 0;
        const u64 m = add_mod(mul_shoup(a, pinv[i], pinv_s[i], q), dd, q);
        u64 r = mul_shoup(sub_mod(m, v, q), tab->qlinv[i], tab->qlinv_s[i], q);
        if (mode == 1) {
            r = add_mod(r, add[(long long)j * add_bs + ((long long)t * add_cap + i) * N + k], q);
        } else if (mode == 2) {
            r = add_mod(r, r, q);
            if (t == 0) r = sub_mod(r, cres[i], q);
        }
        out[(long long)j * out_bs + ((long long)t * out_cap + i) * N + k] = r;
    }
};

// row pass: one CTA = RPC rows of S contiguous elements (RT threads), S/8 threads per row
template <int LOG, int LOGR, bool INV, class E, int RT>
__global__ void __launch_bounds__(RT, RT == 128 ? 9 : 4) k_ntt_row(const __grid_constant__ RingDev R, const __grid_constant__ PolyBatch b,
                                                                   const __grid_constant__ E epi) {
    pdl_wait();
    pdl_trigger();
    constexpr int S = 1 << LOG;
    constexpr int TPR = S / 8;           // threads per row
    constexpr int RPC = (RT / TPR < (1 << LOGR)) ? RT / TPR : (1 << LOGR);  // rows per CTA
    constexpr int SP = S;                // row stride in shared memory (swizzled, no padding)
    extern __shared__ u64 sm[];
    const int N = R.N;
    const int p = blockIdx.y;
    int pi;
    u64* x = poly_at(b, p, N, &pi);
    const u64 q = R.primes[pi].q;
    const ulonglong2* tw = (INV ? R.itw : R.tw) + (size_t)pi * N;
    const int rloc = threadIdx.x / TPR;
    const int tau = threadIdx.x % TPR;
    const int rho = blockIdx.x * RPC + rloc;
    const int Jbase = rho * S;
    u64* xr = x + Jbase;
    const u64* xin = (INV ? poly_in(b, p, N, x) : x) + Jbase;  // the row pass is the inverse's first
    constexpr int L0 = PhaseInfo<LOG, INV, 0>::LO;
    constexpr int LL = LastLo<LOG, INV>::v;
    u64 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = xin[phase_x<L0>(tau, e)];
    const bool grow = q < (1ull << 57);
    Ctx<true> c{Jbase, N, tw, q, grow};
    RowEx ex{sm + rloc * SP};
    phases<LOG, INV, 0>(v, tau, c, ex);
    if constexpr (std::is_same<E, EpiToMont>::value) {
        static_assert(!INV, "epilogues follow forward transforms");
        const DevPrime P = R.primes[pi];
#pragma unroll
        for (int e = 0; e < 8; ++e)
            xr[phase_x<LL>(tau, e)] = to_mont(grow ? mul_shoup(v[e], 1, P.one_s, q) : reduce4(v[e], q), P);
    } else if constexpr (!std::is_same<E, EpiStore>::value) {
        static_assert(!INV, "epilogues follow forward transforms");
        const u64 one_s = R.primes[pi].one_s;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const u64 fv = grow ? mul_shoup(v[e], 1, one_s, q) : reduce4(v[e], q);
            epi.put(p, Jbase + phase_x<LL>(tau, e), fv, q);
        }
    } else if (INV) {
#pragma unroll
        for (int e = 0; e < 8; ++e) xr[phase_x<LL>(tau, e)] = v[e];
    } else if (grow) {
        const u64 one_s = R.primes[pi].one_s;
#pragma unroll
        for (int e = 0; e < 8; ++e) xr[phase_x<LL>(tau, e)] = mul_shoup(v[e], 1, one_s, q);
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) xr[phase_x<LL>(tau, e)] = reduce4(v[e], q);
    }
}

// Single-launch NTT of N = 2^16 (256 x 256) for small batches. A cluster of 8 CTAs of 1024
// threads holds one polynomial, 64 KiB per CTA. Forward: CTA c transforms columns
// [32c, 32c + 32) (column pass, exchanges in buffer A), then writes every result straight
// into the receive buffer (B) of the CTA owning its row block [32r, 32r + 32) through
// distributed shared memory; after the cluster barrier each CTA runs the row pass on its
// 32 rows (exchanges in A) and stores them. Inverse: row pass first (rows from global,
// exchanges in B), results to the column owners' A, then the column pass (exchanges in B).
// The intermediate never goes through global memory and the transform is one launch.
constexpr int kClusterCtas = 8;
constexpr size_t kClusterSmem = (size_t)(2 * 8192 + 2 * 256) * sizeof(u64);

template <bool INV, class E>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(1024, 1)
    k_ntt_cluster(const __grid_constant__ RingDev R, const __grid_constant__ PolyBatch b,
                  const __grid_constant__ E epi) {
    pdl_wait();
    pdl_trigger();
    namespace cg = cooperative_groups;
    constexpr int LOG = 8, S = 256;
    extern __shared__ u64 sm[];
    u64* A = sm;              // 32 rows x 256 (row layout) / 256 rows x 32 columns (column layout)
    u64* Bb = sm + 8192;
    ulonglong2* sw = reinterpret_cast<ulonglong2*>(sm + 16384);  // column-pass twiddles [0, 256)
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int N = R.N;
    const int p = blockIdx.y;
    int pi;
    u64* x = poly_at(b, p, N, &pi);
    const u64 q = R.primes[pi].q;
    const ulonglong2* tw = (INV ? R.itw : R.tw) + (size_t)pi * N;
    for (int i = threadIdx.x; i < S; i += blockDim.x) sw[i] = __ldg(tw + i);
    const bool grow = q < (1ull << 57);
    // column-pass coordinates: column 32 rank + col, rows phase_x(tauc, e)
    const int col = threadIdx.x & 31, tauc = threadIdx.x >> 5;
    const int gcol = rank * 32 + col;
    // row-pass coordinates: row 32 rank + rloc, elements phase_x(taur, e)
    const int rloc = threadIdx.x >> 5, taur = threadIdx.x & 31;
    const int rho = rank * 32 + rloc;
    u64 v[8];
    if constexpr (!INV) {
        constexpr int L0 = PhaseInfo<LOG, false, 0>::LO, LL = LastLo<LOG, false>::v;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = x[(long long)phase_x<L0>(tauc, e) * S + gcol];
        __syncthreads();
        Ctx<false> c{0, S, sw, q, grow};
        ColEx<32> exc{A, col};
        phases<LOG, false, 0>(v, tauc, c, exc);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int row = phase_x<LL>(tauc, e);
            u64* dst = cl.map_shared_rank(Bb, row >> 5);
            dst[(row & 31) * S + gcol] = v[e];
        }
        cl.sync();
        u64* br = Bb + rloc * S;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = br[phase_x<L0>(taur, e)];
        Ctx<true> cr{rho * S, N, tw, q, grow};
        RowEx exr{A + rloc * S};
        phases<LOG, false, 0>(v, taur, cr, exr);
        const u64 one_s = R.primes[pi].one_s;
        u64* xr = x + (long long)rho * S;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const u64 fv = grow ? mul_shoup(v[e], 1, one_s, q) : reduce4(v[e], q);
            if constexpr (std::is_same<E, EpiStore>::value) xr[phase_x<LL>(taur, e)] = fv;
            else if constexpr (std::is_same<E, EpiToMont>::value) xr[phase_x<LL>(taur, e)] = to_mont(fv, R.primes[pi]);
            else epi.put(p, rho * S + phase_x<LL>(taur, e), fv, q);
        }
    } else {
        constexpr int L0 = PhaseInfo<LOG, true, 0>::LO, LL = LastLo<LOG, true>::v;
        const u64* xr = x + (long long)rho * S;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = xr[phase_x<L0>(taur, e)];
        Ctx<true> cr{rho * S, N, tw, q, false};
        RowEx exr{Bb + rloc * S};
        phases<LOG, true, 0>(v, taur, cr, exr);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = phase_x<LL>(taur, e);
            u64* dst = cl.map_shared_rank(A, k >> 5);
            dst[rho * 32 + (k & 31)] = v[e];
        }
        cl.sync();
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = A[phase_x<L0>(tauc, e) * 32 + col];
        Ctx<false> c{0, S, sw, q, false};
        ColEx<32> exc{Bb, col};
        phases<LOG, true, 0>(v, tauc, c, exc);
        const DevPrime P = R.primes[pi];
#pragma unroll
        for (int e = 0; e < 8; ++e)
            x[(long long)phase_x<LL>(tauc, e) * S + gcol] = mul_shoup(v[e], P.ninv, P.ninv_s, q);
    }
}

// ---------------------------------------------------------------------------
// Radix-16 passes for N = 2^16 (tile shape 5): every thread keeps 16 residues and runs 4
// stages per shared-memory exchange, so each 256-point pass is two 4-stage phases with one
// exchange (radix 8: three phases, two exchanges) and a stage on register bit lb loads
// 8 >> lb twiddles for its 8 butterflies. Forward phases take register bits 4..7 then 0..3,
// inverse ones 0..3 then 4..7. Residues whose 16 elements are contiguous in memory move as
// 16-byte vectors.
// ---------------------------------------------------------------------------
template <int LO>
__device__ __forceinline__ int px16(int tau, int e) {
    return ((tau >> LO) << (LO + 4)) | (e << LO) | (tau & ((1 << LO) - 1));
}

template <bool INV, int LO, int B, class C>
__device__ __forceinline__ void stage16(u64 (&v)[16], int tau, const C& c) {
    constexpr int lb = B - LO;
    constexpr int NT = 8 >> lb;
    const u64 q2 = 2 * c.q;
    const int base = (c.M + c.Jbase + ((tau >> LO) << (LO + 4))) >> (B + 1);
    ulonglong2 w[NT];
#pragma unroll
    for (int u = 0; u < NT; ++u) w[u] = c.ld(base + u);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        if (e & (1 << lb)) continue;
        const int e1 = e | (1 << lb);
        const ulonglong2 t = w[e >> (lb + 1)];
        if (!INV) {
            u64 X = v[e];
            if (!c.grow) X = X >= q2 ? X - q2 : X;
            const u64 T = shoup_lazy(v[e1], t.x, t.y, c.q);
            v[e] = X + T;
            v[e1] = X - T + q2;
        } else {
            const u64 X = v[e], Y = v[e1];
            u64 S = X + Y;
            S = S >= q2 ? S - q2 : S;
            v[e] = S;
            v[e1] = shoup_lazy(X - Y + q2, t.x, t.y, c.q);
        }
    }
}

// the four stages of a phase whose register bits start at LO: forward bits LO+3 .. LO,
// inverse LO .. LO+3
template <bool INV, int LO, class C>
__device__ __forceinline__ void phase16(u64 (&v)[16], int tau, const C& c) {
    if constexpr (!INV) {
        stage16<false, LO, LO + 3>(v, tau, c);
        stage16<false, LO, LO + 2>(v, tau, c);
        stage16<false, LO, LO + 1>(v, tau, c);
        stage16<false, LO, LO>(v, tau, c);
    } else {
        stage16<true, LO, LO>(v, tau, c);
        stage16<true, LO, LO + 1>(v, tau, c);
        stage16<true, LO, LO + 2>(v, tau, c);
        stage16<true, LO, LO + 3>(v, tau, c);
    }
}

// Shared-memory word of element x of a 256-point row: x ^ ((x >> 4) & 15). A half-warp (one
// row's 16 threads) then touches 16 distinct 8-byte bank pairs both when it stores elements
// e << 4 | tau and when it loads tau << 4 | e (and the reverse).
__device__ __forceinline__ int sw16(int x) { return x ^ ((x >> 4) & 15); }

// column pass: one CTA = 8 columns x 256 rows, thread (tau, col) = (threadIdx / 8, threadIdx % 8)
template <bool INV>
__global__ void __launch_bounds__(128, 4) k_ntt_col16(const __grid_constant__ RingDev R,
                                                      const __grid_constant__ PolyBatch b) {
    pdl_wait();
    pdl_trigger();
    constexpr int S = 256, KTC = 8;
    extern __shared__ u64 sm[];                                    // [S][KTC] rows swizzled
    ulonglong2* sw = reinterpret_cast<ulonglong2*>(sm + S * KTC);  // twiddles [0, S)
    const int N = R.N;
    const int C = N >> 8;
    const int p = blockIdx.y;
    int pi;
    u64* x = poly_at(b, p, N, &pi);
    const u64 q = R.primes[pi].q;
    const ulonglong2* tw = (INV ? R.itw : R.tw) + (size_t)pi * N;
    for (int i = threadIdx.x; i < S; i += blockDim.x) sw[i] = __ldg(tw + i);
    const int col = threadIdx.x & (KTC - 1);
    const int tau = threadIdx.x / KTC;
    const int gcol = blockIdx.x * KTC + col;
    constexpr int L0 = INV ? 0 : 4, L1 = INV ? 4 : 0;
    u64 v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = x[(long long)px16<L0>(tau, e) * C + gcol];
    __syncthreads();
    Ctx<false> c{0, S, sw, q, q < (1ull << 57)};
    phase16<INV, L0>(v, tau, c);
    // rows x and x + 16 of one load phase fall in different bank halves: row' = x ^ bit 4 of x
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int r = px16<L0>(tau, e);
        sm[(r ^ ((r >> 4) & 1)) * KTC + col] = v[e];
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int r = px16<L1>(tau, e);
        v[e] = sm[(r ^ ((r >> 4) & 1)) * KTC + col];
    }
    phase16<INV, L1>(v, tau, c);
    if (INV) {
        const DevPrime P = R.primes[pi];
#pragma unroll
        for (int e = 0; e < 16; ++e)
            x[(long long)px16<L1>(tau, e) * C + gcol] = mul_shoup(v[e], P.ninv, P.ninv_s, q);
    } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) x[(long long)px16<L1>(tau, e) * C + gcol] = v[e];
    }
}

// row pass: one CTA = 8 rows of 256 contiguous elements, 16 threads per row
template <bool INV, class E>
__global__ void __launch_bounds__(128, 4) k_ntt_row16(const __grid_constant__ RingDev R,
                                                      const __grid_constant__ PolyBatch b,
                                                      const __grid_constant__ E epi) {
    pdl_wait();
    pdl_trigger();
    constexpr int S = 256, TPR = 16, RPC = 8;
    extern __shared__ u64 sm[];  // [RPC][S] swizzled
    const int N = R.N;
    const int p = blockIdx.y;
    int pi;
    u64* x = poly_at(b, p, N, &pi);
    const u64 q = R.primes[pi].q;
    const ulonglong2* tw = (INV ? R.itw : R.tw) + (size_t)pi * N;
    const int rloc = threadIdx.x / TPR;
    const int tau = threadIdx.x % TPR;
    const int rho = blockIdx.x * RPC + rloc;
    const int Jbase = rho * S;
    u64* xr = x + Jbase;
    constexpr int L0 = INV ? 0 : 4, L1 = INV ? 4 : 0;
    u64 v[16];
    if constexpr (L0 == 0) {
        // the thread's 16 elements are contiguous: eight 16-byte loads
        const ulonglong2* src = reinterpret_cast<const ulonglong2*>(xr + tau * 16);
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const ulonglong2 t = src[h];
            v[2 * h] = t.x;
            v[2 * h + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = xr[px16<L0>(tau, e)];
    }
    const bool grow = q < (1ull << 57);
    Ctx<true> c{Jbase, N, tw, q, INV ? false : grow};
    phase16<INV, L0>(v, tau, c);
    u64* s = sm + rloc * S;
#pragma unroll
    for (int e = 0; e < 16; ++e) s[sw16(px16<L0>(tau, e))] = v[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = s[sw16(px16<L1>(tau, e))];
    phase16<INV, L1>(v, tau, c);
    if constexpr (INV) {
#pragma unroll
        for (int e = 0; e < 16; ++e) xr[px16<L1>(tau, e)] = v[e];
    } else {
        const u64 one_s = R.primes[pi].one_s;
        u64 o[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) o[e] = grow ? mul_shoup(v[e], 1, one_s, q) : reduce4(v[e], q);
        if constexpr (std::is_same<E, EpiStore>::value) {
            ulonglong2* dst = reinterpret_cast<ulonglong2*>(xr + tau * 16);
#pragma unroll
            for (int h = 0; h < 8; ++h) dst[h] = make_ulonglong2(o[2 * h], o[2 * h + 1]);
        } else if constexpr (std::is_same<E, EpiToMont>::value) {
            const DevPrime P = R.primes[pi];
            ulonglong2* dst = reinterpret_cast<ulonglong2*>(xr + tau * 16);
#pragma unroll
            for (int h = 0; h < 8; ++h) dst[h] = make_ulonglong2(to_mont(o[2 * h], P), to_mont(o[2 * h + 1], P));
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) epi.put(p, Jbase + tau * 16 + e, o[e], q);
        }
    }
}

template <class E>
void launch_ntt_r16(const RingDev& R, const PolyBatch& b, bool inverse, cudaStream_t st, const E& epi) {
    const int N = R.N;
    const dim3 gc((N >> 8) / 8, b.npolys), gr(256 / 8, b.npolys);
    const size_t smc = (size_t)(256 * 8 + 2 * 256) * sizeof(u64), smr = (size_t)8 * 256 * sizeof(u64);
    if (!inverse) {
        launch_k(k_ntt_col16<false>, gc, dim3(128), smc, st, R, b);
        launch_k(k_ntt_row16<false, E>, gr, dim3(128), smr, st, R, b, epi);
    } else {
        launch_k(k_ntt_row16<true, EpiStore>, gr, dim3(128), smr, st, R, b, EpiStore{});
        launch_k(k_ntt_col16<true>, gc, dim3(128), smc, st, R, b);
    }
}

template <int LOGR, int LOGC, class E, int KTC, int RT>
void launch_ntt_t(const RingDev& R, const PolyBatch& b, bool inverse, cudaStream_t st, const E& epi) {
    constexpr int SR = 1 << LOGR, SC = 1 << LOGC;
    const int N = R.N;
    dim3 gc((N >> LOGR) / KTC, b.npolys);
    const int tc = KTC * SR / 8;
    const size_t smc = (size_t)(SR * KTC + 2 * SR) * sizeof(u64);
    constexpr int TPR = SC / 8, RPC = (RT / TPR < SR) ? RT / TPR : SR;
    dim3 gr(SR / RPC, b.npolys);
    const size_t smr = (size_t)RPC * SC * sizeof(u64);
    if (!inverse) {
        launch_k(k_ntt_col<LOGR, false, KTC>, dim3(gc), dim3(tc), smc, st, R, b);
        launch_k(k_ntt_row<LOGC, LOGR, false, E, RT>, dim3(gr), dim3(RPC * TPR), smr, st, R, b, epi);
    } else {
        launch_k(k_ntt_row<LOGC, LOGR, true, EpiStore, RT>, dim3(gr), dim3(RPC * TPR), smr, st, R, b, EpiStore{});
        launch_k(k_ntt_col<LOGR, true, KTC>, dim3(gc), dim3(tc), smc, st, R, b);
    }
}

// Tile shape of a launch: 0..3 are the radix-8 two-pass kernels, bit 0 set = 8 columns per
// column-pass CTA (else 4), bit 1 set = 256-thread row-pass CTAs (else 128); 4 is the
// single-launch cluster kernel and 5 the radix-16 two-pass kernels (both N = 2^16). Chosen per
// batch-size bucket by the tuner (RingDev holds the table); sizes other than N = 2^15, 2^16
// use shape 0.
template <class E>
void launch_ntt_cluster(const RingDev& R, const PolyBatch& b, bool inverse, cudaStream_t st, const E& epi) {
    static std::atomic<unsigned long long> fwd{0}, inv{0};
    smem_limit_once(k_ntt_cluster<false, E>, (int)kClusterSmem, fwd);
    smem_limit_once(k_ntt_cluster<true, EpiStore>, (int)kClusterSmem, inv);
    const dim3 g(kClusterCtas, b.npolys);
    if (!inverse) launch_k(k_ntt_cluster<false, E>, g, dim3(1024), kClusterSmem, st, R, b, epi);
    else launch_k(k_ntt_cluster<true, EpiStore>, g, dim3(1024), kClusterSmem, st, R, b, EpiStore{});
}

template <int LOGR, int LOGC, class E>
void launch_ntt_s(const RingDev& R, const PolyBatch& b, bool inverse, cudaStream_t st, const E& epi) {
    const int shape = (LOGR + LOGC >= 15) ? R.ntt_shape[ntt_bucket(b.npolys)] : 0;
    if constexpr (LOGR == 8 && LOGC == 8) {
        if (shape == 4) {
            launch_ntt_cluster(R, b, inverse, st, epi);
            return;
        }
        if (shape == 5) {
            launch_ntt_r16(R, b, inverse, st, epi);
            return;
        }
    }
    switch (shape) {
        case 1: launch_ntt_t<LOGR, LOGC, E, 8, 128>(R, b, inverse, st, epi); break;
        case 2: launch_ntt_t<LOGR, LOGC, E, 4, 256>(R, b, inverse, st, epi); break;
        case 3: launch_ntt_t<LOGR, LOGC, E, 8, 256>(R, b, inverse, st, epi); break;
        default: launch_ntt_t<LOGR, LOGC, E, 4, 128>(R, b, inverse, st, epi); break;
    }
}

// Register-only throughput of the forward butterfly used above (Harvey lazy reduction,
// Shoup twiddle product): the arithmetic ceiling of the NTT on this GPU, no memory traffic.
__global__ void __launch_bounds__(256) k_butterfly_peak(u64 q, u64 w, u64 ws, int iters, u64* sink) {
    u64 x[8], y[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        x[e] = (threadIdx.x * 8 + e) % q;
        y[e] = (blockIdx.x * 8 + e + 1) % q;
    }
    const u64 q2 = 2 * q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            u64 X = x[e];
            X = X >= q2 ? X - q2 : X;
            const u64 T = shoup_lazy(y[e], w, ws, q);
            x[e] = X + T;
            y[e] = X - T + q2;
        }
    }
    u64 acc = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) acc ^= x[e] ^ y[e];
    if (acc == 0x5a5a5a5a5a5a5a5aull) sink[0] = acc;  // keeps the loop live
}

}  // namespace

int pdl_mode() {
    static const int m = [] {
        const char* e = std::getenv("FR_PDL");
        return e && e[0] == '0' ? 0 : e && e[0] == '1' ? 1 : 2;
    }();
    return m;
}

double measure_butterfly_peak(int device) {
    // 60-bit prime; any twiddle works for a throughput measurement
    const u64 q = 1152921504606830593ull, w = 0x0123456789abcdefull % q;
    const u64 ws = (u64)(((unsigned __int128)w << 64) / q);
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    u64* sink = nullptr;
    if (cudaMalloc(&sink, 8) != cudaSuccess) return 0;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_butterfly_peak<<<blocks, threads>>>(q, w, ws, 64, sink);  // warm-up
    cudaEventRecord(a);
    k_butterfly_peak<<<blocks, threads>>>(q, w, ws, iters, sink);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    if (ms <= 0) return 0;
    return (double)blocks * threads * 8.0 * iters / (ms * 1e-3);
}

template <class E>
void launch_ntt_e(const RingDev& R, const PolyBatch& b, bool inverse, cudaStream_t s, const E& epi) {
    if (b.npolys <= 0) return;
    if (b.src) {
        // the radix-8 two-pass kernels read a source themselves; for the cluster and radix-16
        // shapes (and a table-mapped batch) the source is copied into place first
        const int shape = R.logN >= 15 ? R.ntt_shape[ntt_bucket(b.npolys)] : 0;
        if (b.tab || shape == 4 || shape == 5) {
            cudaMemcpy2DAsync(b.base, (size_t)b.outer * 8, b.src, (size_t)b.src_outer * 8, (size_t)b.inner * R.N * 8,
                              (size_t)(b.npolys / b.inner), cudaMemcpyDeviceToDevice, s);
            PolyBatch c = b;
            c.src = nullptr;
            launch_ntt_e(R, c, inverse, s, epi);
            return;
        }
    }
    switch (R.logN) {
        case 10: launch_ntt_t<5, 5, E, 4, 128>(R, b, inverse, s, epi); break;
        case 11: launch_ntt_t<5, 6, E, 4, 128>(R, b, inverse, s, epi); break;
        case 12: launch_ntt_t<6, 6, E, 4, 128>(R, b, inverse, s, epi); break;
        case 13: launch_ntt_t<6, 7, E, 4, 128>(R, b, inverse, s, epi); break;
        case 14: launch_ntt_t<7, 7, E, 4, 128>(R, b, inverse, s, epi); break;
        case 15: launch_ntt_s<7, 8, E>(R, b, inverse, s, epi); break;
        case 16: launch_ntt_s<8, 8, E>(R, b, inverse, s, epi); break;
        default: break;
    }
}

void launch_ntt(const RingDev& R, const PolyBatch& b, bool inverse, cudaStream_t s) {
    launch_ntt_e(R, b, inverse, s, EpiStore{});
}

// Times every tile shape of the forward + inverse transform for one batch size per bucket
// (CUDA events, best of `reps`) on a scratch buffer of zero residues and keeps the fastest
// shape per bucket in R.ntt_shape; us[bucket * 4 + shape] receives the times.
void tune_ntt(RingDev& R, cudaStream_t s, double* us, int reps) {
    for (int bk = 0; bk < FR_NTT_BUCKETS; ++bk) R.ntt_shape[bk] = 0;
    if (us)
        for (int i = 0; i < FR_NTT_BUCKETS * FR_NTT_SHAPES; ++i) us[i] = 0;
    if (R.logN < 15) return;
    const int nshapes = R.logN == 16 ? FR_NTT_SHAPES : FR_NTT_SHAPES - 2;  // shapes 4 and 5 are N = 2^16 only
    const int sizes[FR_NTT_BUCKETS] = {4, 16, 64, 256};
    const int maxp = sizes[FR_NTT_BUCKETS - 1];
    u64* buf = nullptr;
    if (cudaMallocAsync(&buf, (size_t)maxp * R.N * 8, s) != cudaSuccess) { cudaGetLastError(); return; }
    cudaMemsetAsync(buf, 0, (size_t)maxp * R.N * 8, s);
    cudaEvent_t a, e;
    cudaEventCreate(&a);
    cudaEventCreate(&e);
    unsigned char best[FR_NTT_BUCKETS];
    for (int bk = 0; bk < FR_NTT_BUCKETS; ++bk) {
        PolyBatch pb{buf, 0, sizes[bk], sizes[bk], PrimeMap{}};
        pb.pm.period = 1;
        pb.pm.idx[0] = 0;
        double tbest = 1e30, t0 = 1e30;
        best[bk] = 0;
        for (int sh = 0; sh < nshapes; ++sh) {
            R.ntt_shape[bk] = (unsigned char)sh;
            double t = 1e30;
            for (int r = 0; r <= reps; ++r) {  // first run warms up
                cudaEventRecord(a, s);
                launch_ntt(R, pb, false, s);
                launch_ntt(R, pb, true, s);
                cudaEventRecord(e, s);
                cudaEventSynchronize(e);
                float ms = 0;
                cudaEventElapsedTime(&ms, a, e);
                if (r > 0) t = t < ms * 1000.0 ? t : ms * 1000.0;
            }
            if (cudaGetLastError() != cudaSuccess) t = 1e30;  // a shape this GPU cannot launch
            if (us) us[bk * FR_NTT_SHAPES + sh] = t < 1e29 ? t : -1.0;
            // another shape replaces the default only when at least 3% faster (timing noise)
            if (sh == 0) t0 = t;
            if (sh == 0 ? t < tbest : t < tbest && t < 0.97 * t0) {
                tbest = t;
                best[bk] = (unsigned char)sh;
            }
        }
    }
    for (int bk = 0; bk < FR_NTT_BUCKETS; ++bk) R.ntt_shape[bk] = best[bk];
    cudaEventDestroy(a);
    cudaEventDestroy(e);
    cudaFreeAsync(buf, s);
    cudaStreamSynchronize(s);
}

void launch_ntt_tomont(const RingDev& R, const PolyBatch& b, cudaStream_t s) {
    launch_ntt_e(R, b, false, s, EpiToMont{});
}

void launch_ntt_moddown(const RingDev& R, const PolyBatch& b, const MDJobs& jobs, int npos, int level,
                        const u64* pinv, const u64* pinv_s, cudaStream_t s) {
    EpiModDown e{jobs, npos, level, R.logN, pinv, pinv_s};
    launch_ntt_e(R, b, false, s, e);
}

void launch_ntt_relin_rescale(const RingDev& R, const PolyBatch& b, const u64* acc, const u64* d, int npos, int l,
                              const u64* pinv, const u64* pinv_s, const RescaleTab* tab, u64* out, int out_cap,
                              long long out_bs, int mode, const u64* add, int add_cap, long long add_bs,
                              const u64* cres, cudaStream_t s) {
    EpiRelinRescale e{acc, d, out, tab, pinv, pinv_s, npos, l, R.N, out_cap, mode, out_bs, add, add_cap, add_bs, cres};
    launch_ntt_e(R, b, false, s, e);
}

void launch_ntt_leaf_rescale(const RingDev& R, const PolyBatch& b, const u64* x, long long x_bs, int x_cap,
                             const u64* cb, const u64* cb_s, const u64* ca, int nl, int L1, u64* out, int out_cap,
                             const RescaleTab* tab, int l, cudaStream_t s) {
    EpiLeafRescale e{x, x_bs, x_cap, cb, cb_s, ca, nl, L1, out, out_cap, tab, l, R.N};
    launch_ntt_e(R, b, false, s, e);
}

void launch_ntt_rescale(const RingDev& R, const PolyBatch& b, const u64* x, int x_cap, u64* out, int out_cap,
                        const RescaleTab* tab, int l, int mode, const u64* add, int add_cap, long long add_bs,
                        const u64* cres, cudaStream_t s) {
    EpiRescale e{x, out, tab, x_cap, out_cap, l, R.N, mode, add, add_cap, add_bs, cres};
    launch_ntt_e(R, b, false, s, e);
}
