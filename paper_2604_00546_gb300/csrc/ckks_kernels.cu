// CKKS device kernels: base conversion (ModUp / ModDown), key-switch inner
// product with the slot automorphism fused into its gather, rescale, tensor
// product, the diagonal plaintext x ciphertext multiply-accumulate, Chebyshev
// scalar steps and the on-device slot encoder for template diagonals.
#include <algorithm>
#include <cstdio>

#include "ckks_kernels.h"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void fold(Acc128& a, u64 q) {
    if (a.hi >= q) a.hi -= q;
}

// ---------------------------------------------------------------------------
// ModUp: per digit, fast-convert the digit's limbs to every other position of
// Q_l u P (coefficient form); the digit's own positions are copied from the
// evaluation-form input so they need no forward NTT afterwards.
// in: coefficient form, job j at in + j * in_job; in_eval: evaluation form, job j at in_eval + j * eval_job
// ext: [J][beta][npos][N]
// ---------------------------------------------------------------------------
// sum_i ys_i [B/b_i]_t mod t from split residues: 30-bit multiply-accumulate, the high word
// reduced mod t, then one Montgomery reduction (hat_m carries the 2^64 factor)
template <int NS>
__device__ __forceinline__ u64 bconv_sum(const u64 (&ys)[NS], const u64 (&hat_m)[FR_MAX_DIGIT_LIMBS][FR_MAX_PRIMES],
                                         int pos, u64 t, u64 tinv, u64 t_one_s) {
    AccK a{0, 0, 0};
#pragma unroll
    for (int i = 0; i < NS; ++i) mack(a, ys[i], sum30(ys[i]), hat_m[i][pos]);
    Acc128 acc{0, 0};
    flushk(acc, a);
    return redc(mul_shoup(acc.hi, 1, t_one_s, t), acc.lo, t, tinv);
}

template <int NS>
__device__ __forceinline__ void modup_body(const ModUpTab& T, const u64* __restrict__ x,
                                           const u64* __restrict__ xe, u64* __restrict__ out, int npos, int N,
                                           int k) {
    u64 ys[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i)
        ys[i] = split30(mul_shoup(x[(long long)(T.lo + i) * N + k], T.inv_hat[i], T.inv_hat_s[i], T.src_q[i]));
    for (int pos = 0; pos < npos; ++pos) {
        u64 v;
        if (pos >= T.lo && pos < T.lo + NS) v = xe[(long long)pos * N + k];
        else v = bconv_sum<NS>(ys, T.hat_m, pos, T.tq[pos], T.tinv[pos], T.t_one_s[pos]);
        out[(long long)pos * N + k] = v;
    }
}

__global__ void __launch_bounds__(kThreads) k_modup(const u64* __restrict__ in, long long in_job,
                                                    const u64* __restrict__ in_eval, long long eval_job,
                                                    u64* __restrict__ ext, const ModUpTab* __restrict__ tabs, int beta,
                                                    int npos, int N) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    const int j = blockIdx.z;
    if (k >= N) return;
    const ModUpTab& T = tabs[d];
    const u64* x = in + (long long)j * in_job;
    const u64* xe = in_eval + (long long)j * eval_job;
    u64* out = ext + (((long long)j * beta + d) * npos) * N;
    switch (T.ns) {
        case 1: modup_body<1>(T, x, xe, out, npos, N, k); break;
        case 2: modup_body<2>(T, x, xe, out, npos, N, k); break;
        case 3: modup_body<3>(T, x, xe, out, npos, N, k); break;
        case 4: modup_body<4>(T, x, xe, out, npos, N, k); break;
        case 5: modup_body<5>(T, x, xe, out, npos, N, k); break;
        case 6: modup_body<6>(T, x, xe, out, npos, N, k); break;
        case 7: modup_body<7>(T, x, xe, out, npos, N, k); break;
        default: modup_body<8>(T, x, xe, out, npos, N, k); break;  // ns <= 8, checked on the host
    }
}

// ---------------------------------------------------------------------------
// Key-switch inner product: acc_t[pos] = sum_d sigma_g(ext_d[pos]) * key_d[t][limb(pos)]
// Keys are stored in Montgomery form, so one REDC of the 128-bit sum gives
// the canonical residue. The automorphism is a gather on the ext index. When
// all jobs of a launch use the same key (batched relinearisation), a thread
// reads its key words once and applies them to every job.
// ---------------------------------------------------------------------------
template <int BETA>
__device__ __forceinline__ void ip_job(const IPJob& J, const u64 (&k0)[BETA], const u64 (&k1)[BETA], int npos, int pos,
                                       int k, u64 q, u64 qinv, int logN, int N, int level, const u64* pmod,
                                       const u64* pmod_s) {
    const u32 src = J.galois != 1u ? galois_src_index((u32)k, J.galois, logN) : (u32)k;
    Acc128 a0{0, 0}, a1{0, 0};
#pragma unroll
    for (int d = 0; d < BETA; ++d) {
        const u64 e = J.ext[((long long)d * npos + pos) * N + src];
        mac128(a0, e, k0[d]);
        mac128(a1, e, k1[d]);
        if ((d & 7) == 7) { fold(a0, q); fold(a1, q); }
    }
    fold(a0, q);
    fold(a1, q);
    u64 r0 = redc(a0.hi, a0.lo, q, qinv);
    if (J.addb && pos <= level)  // a rotation kept in Q_l u P: + P sigma(b) on the Q positions
        r0 = add_mod(r0, mul_shoup(J.addb[(long long)pos * N + src], pmod[pos], pmod_s[pos], q), q);
    J.out[(long long)pos * N + k] = r0;
    J.out[((long long)npos + pos) * N + k] = redc(a1.hi, a1.lo, q, qinv);
}

template <int BETA>
__device__ __forceinline__ void ip_body(const IPJobs& jobs, int npos, int pos, int klimb, int T, int k, u64 q,
                                        u64 qinv, int logN, int N, int level, const u64* pmod, const u64* pmod_s) {
    // one key group per blockIdx.y: its key words are read once and applied to every job of the group
    const int g = blockIdx.y;
    const u64* key = jobs.gkey[g];
    u64 k0[BETA], k1[BETA];
#pragma unroll
    for (int d = 0; d < BETA; ++d) {
        k0[d] = key[(((long long)d * 2 + 0) * T + klimb) * N + k];
        k1[d] = key[(((long long)d * 2 + 1) * T + klimb) * N + k];
    }
    for (int j = jobs.gstart[g]; j < jobs.gstart[g + 1]; ++j)
        ip_job<BETA>(jobs.j[j], k0, k1, npos, pos, k, q, qinv, logN, N, level, pmod, pmod_s);
}

// key layout [digit][2][T][N]: Q limbs at positions 0.., P limbs from position kp. One
// instantiation per digit count, so the registers a launch needs follow its beta.
template <int BETA>
__global__ void __launch_bounds__(kThreads) k_ip(const __grid_constant__ IPJobs jobs, int npos, int level, int kp,
                                                 int T, const DevPrime* __restrict__ primes, int pbase, int logN,
                                                 const u64* __restrict__ pmod, const u64* __restrict__ pmod_s) {
    pdl_wait();
    pdl_trigger();
    const int N = 1 << logN;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    // position-major grid: the key groups of one position run back to back, so a ModUp
    // extension that several groups gather from (hoisted rotations) is read from L2
    const int pos = blockIdx.z;
    if (k >= N) return;
    // positions 0..level are Q limbs 0..level; the P limbs follow (prime indices from pbase)
    const int pi = pos <= level ? pos : pbase + (pos - (level + 1));
    const u64 q = primes[pi].q, qinv = primes[pi].qinv;
    const int klimb = pos <= level ? pos : kp + (pos - (level + 1));
    ip_body<BETA>(jobs, npos, pos, klimb, T, k, q, qinv, logN, N, level, pmod, pmod_s);
}

// Inner products summed into their accumulator (double-hoisted sums of rotations): thread
// (point k, group g, position pos) runs the jobs of group g, each a key-switch inner product
// of its ext under its automorphism (the same products as ip_job), in one 128-bit sum per
// component, folded after every job: a product of two residues below q < 2^61 adds less than
// q/8 to the high word, so a job's beta <= 8 products leave it below 2q before the fold. Then
// it adds P sigma_j(addb_j) on the Q positions of component 0 and the value already in the
// accumulator. The grid is (points, groups, positions), groups fastest after the points:
// the key words of one position, which every group's job with that key reads, are L2 hits
// after the first group.
template <int BETA>
__global__ void __launch_bounds__(kThreads) k_ip_sum(const __grid_constant__ IPSumJobs jobs, int npos, int level,
                                                     int kp, int T, const DevPrime* __restrict__ primes, int pbase,
                                                     int logN, const u64* __restrict__ pmod,
                                                     const u64* __restrict__ pmod_s) {
    pdl_wait();
    pdl_trigger();
    const int N = 1 << logN;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = blockIdx.y;
    const int pos = blockIdx.z;
    if (k >= N) return;
    const int pi = pos <= level ? pos : pbase + (pos - (level + 1));
    const u64 q = primes[pi].q, qinv = primes[pi].qinv;
    const int klimb = pos <= level ? pos : kp + (pos - (level + 1));
    Acc128 a0{0, 0}, a1{0, 0};
    u64 badd = 0;
    for (int jj = jobs.gstart[g]; jj < jobs.gstart[g + 1]; ++jj) {
        const IPJob& J = jobs.j[jj];
        const u32 src = J.galois != 1u ? galois_src_index((u32)k, J.galois, logN) : (u32)k;
#pragma unroll
        for (int d = 0; d < BETA; ++d) {
            const u64 e = J.ext[((long long)d * npos + pos) * N + src];
            mac128(a0, e, J.key[(((long long)d * 2 + 0) * T + klimb) * N + k]);
            mac128(a1, e, J.key[(((long long)d * 2 + 1) * T + klimb) * N + k]);
        }
        fold(a0, q);
        fold(a1, q);
        if (J.addb && pos <= level)
            badd = add_mod(badd, mul_shoup(J.addb[(long long)pos * N + src], pmod[pos], pmod_s[pos], q), q);
    }
    u64* O = jobs.j[jobs.gstart[g]].out;
    const long long o0 = (long long)pos * N + k, o1 = ((long long)npos + pos) * N + k;
    O[o0] = add_mod(O[o0], add_mod(redc(a0.hi, a0.lo, q, qinv), badd, q), q);
    O[o1] = add_mod(O[o1], redc(a1.hi, a1.lo, q, qinv), q);
}

// ---------------------------------------------------------------------------
// ModDown base conversion P -> Q_l of the (coefficient-form) P limbs of acc.
// acc: job j at acc + j * acc_job, poly t at + t * npos * N, P limb jj at position level+1+jj
// conv: [J][2][level+1][N]
// ---------------------------------------------------------------------------
template <int NP>
__device__ __forceinline__ void p2q_body(const u64* __restrict__ x, u64* __restrict__ o, const P2QTab* __restrict__ tab,
                                         int level, int N, int k) {
    u64 ys[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i)
        ys[i] = split30(mul_shoup(x[(long long)(level + 1 + i) * N + k], tab->inv_hat[i], tab->inv_hat_s[i], tab->pq[i]));
    for (int i = 0; i <= level; ++i)
        o[(long long)i * N + k] = bconv_sum<NP>(ys, tab->hat_m, i, tab->qq[i], tab->qinv[i], tab->q_one_s[i]);
}

__global__ void __launch_bounds__(kThreads) k_p2q(const u64* __restrict__ acc, long long acc_job, int npos,
                                                  int level, u64* __restrict__ conv, const P2QTab* __restrict__ tab,
                                                  int N) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    const int j = blockIdx.z;
    if (k >= N) return;
    const u64* x = acc + (long long)j * acc_job + (long long)t * npos * N;
    u64* o = conv + ((long long)j * 2 + t) * (level + 1) * N;
    switch (tab->np) {
        case 1: p2q_body<1>(x, o, tab, level, N, k); break;
        case 2: p2q_body<2>(x, o, tab, level, N, k); break;
        case 3: p2q_body<3>(x, o, tab, level, N, k); break;
        case 4: p2q_body<4>(x, o, tab, level, N, k); break;
        case 5: p2q_body<5>(x, o, tab, level, N, k); break;
        case 6: p2q_body<6>(x, o, tab, level, N, k); break;
        case 7: p2q_body<7>(x, o, tab, level, N, k); break;
        default: p2q_body<8>(x, o, tab, level, N, k); break;  // np <= 8, checked on the host
    }
}

// out[t][i] = (acc[t][i] - conv[t][i]) * P^-1 + addend   (evaluation form)
// addend modes: 0 none, 1 rotation (t=0 gets sigma_g(add c0)), 2 plain ct add (both polys)
__global__ void __launch_bounds__(kThreads) k_moddown_combine(const MDJobs jobs, int npos, int level,
                                                              const u64* __restrict__ pinv,
                                                              const u64* __restrict__ pinv_s,
                                                              const DevPrime* __restrict__ primes, int logN) {
    pdl_wait();
    pdl_trigger();
    const int N = 1 << logN;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y % (level + 1);
    const int t = blockIdx.y / (level + 1);
    const MDJob& J = jobs.j[blockIdx.z];
    if (k >= N) return;
    const u64 q = primes[i].q;
    const u64 a = J.acc[((long long)t * npos + i) * N + k];
    const u64 c = J.conv[((long long)t * (level + 1) + i) * N + k];
    u64 v = mul_shoup(sub_mod(a, c, q), pinv[i], pinv_s[i], q);
    if (J.mode == 1) {
        if (t == 0) {
            const u32 src = galois_src_index((u32)k, J.galois, logN);
            v = add_mod(v, J.add[(long long)i * N + src], q);
        }
    } else if (J.mode == 2) {
        v = add_mod(v, J.add[((long long)t * J.add_cap + i) * N + k], q);
    }
    J.out[((long long)t * J.out_cap + i) * N + k] = v;
}

// ---------------------------------------------------------------------------
// Rescale. lift: centered last limb (coefficient form) to each q_i, i < l.
// last: [B][2][N] ; lifted: [B][2][l][N]
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_rescale_lift(const u64* __restrict__ last, u64* __restrict__ lifted,
                                                           const RescaleTab* __restrict__ tab, int l, int N) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int bt = blockIdx.y;
    if (k >= N) return;
    const u64 x = last[(long long)bt * N + k];
    const bool neg = x > tab->half;
    u64* o = lifted + (long long)bt * l * N;
    for (int i = 0; i < l; ++i) {
        const u64 q = tab->q[i];
        u64 r = mul_shoup(x, 1, tab->one_s[i], q);  // x mod q
        if (neg) r = sub_mod(r, tab->ql_mod[i], q);
        o[(long long)i * N + k] = r;
    }
}

// Baby steps kept in Q_l u P (double hoisting of the baby steps): baby 0 of query b is P q_b on
// the Q positions and zero on the P positions (babies 1..n1-1 come from the inner-product
// kernel, which adds P sigma_i(q_b.b) itself). babies [B][n1][2][npos][N] (query b at babies +
// b baby_q); q_b at q + b q_bs, [2][q_cap][N], evaluation form. Grid (N / 256, npos, 2 B).
__global__ void __launch_bounds__(kThreads) k_baby0_pq(u64* __restrict__ babies, long long baby_q,
                                                       const u64* __restrict__ q, long long q_bs, int q_cap, int npos,
                                                       int level, const DevPrime* __restrict__ primes,
                                                       const u64* __restrict__ pmod, const u64* __restrict__ pmod_s,
                                                       int N) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int pos = blockIdx.y;
    const int t = blockIdx.z & 1, b = blockIdx.z >> 1;
    if (k >= N) return;
    u64* o = babies + (long long)b * baby_q + ((long long)t * npos + pos) * N + k;
    if (pos > level) {
        *o = 0;
        return;
    }
    const u64 qp = primes[pos].q;
    *o = mul_shoup(q[(long long)b * q_bs + ((long long)t * q_cap + pos) * N + k], pmod[pos], pmod_s[pos], qp);
}

// Relinearisation + rescale, last limb: z = acc_l P^-1 + d_l (evaluation form), the last limb
// of the relinearised product before the rescale. acc [J][2][npos][N], d [J][3][l+1][N] or
// null (a ModDown with no addend), z [J][2][N].
__global__ void __launch_bounds__(kThreads) k_rs_last(const u64* __restrict__ acc, const u64* __restrict__ d,
                                                      u64* __restrict__ z, const u64* __restrict__ pinv,
                                                      const u64* __restrict__ pinv_s, int npos, int l,
                                                      const DevPrime* __restrict__ primes, int N) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int jt = blockIdx.y, j = jt >> 1, t = jt & 1;
    if (k >= N) return;
    const u64 q = primes[l].q;
    const u64 a = acc[((long long)jt * npos + l) * N + k];
    const u64 dd = d ? d[(((long long)j * 3 + t) * (l + 1) + l) * N + k] : 0;
    z[(long long)jt * N + k] = add_mod(mul_shoup(a, pinv[l], pinv_s[l], q), dd, q);
}

// Relinearisation + rescale, lift: with zc = z in coefficient form and conv the P -> Q
// conversion (coefficient form, [J][2][l+1][N]), the relinearised product's last limb is
// m = zc - conv_l P^-1 (mod q_l); y_i = conv_i P^-1 + [centered m]_{q_i} for i < l, [J][2][l][N].
__global__ void __launch_bounds__(kThreads) k_rs_lift(const u64* __restrict__ zc, const u64* __restrict__ conv,
                                                      u64* __restrict__ y, const u64* __restrict__ pinv,
                                                      const u64* __restrict__ pinv_s,
                                                      const RescaleTab* __restrict__ tab,
                                                      const DevPrime* __restrict__ primes, int l, int N) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int jt = blockIdx.y;
    if (k >= N) return;
    const u64 ql = primes[l].q;
    const u64* cv = conv + (long long)jt * (l + 1) * N;
    const u64 m = sub_mod(zc[(long long)jt * N + k], mul_shoup(cv[(long long)l * N + k], pinv[l], pinv_s[l], ql), ql);
    const bool neg = m > tab->half;
    u64* o = y + (long long)jt * l * N;
    for (int i = 0; i < l; ++i) {
        const u64 q = tab->q[i];
        u64 r = mul_shoup(m, 1, tab->one_s[i], q);
        if (neg) r = sub_mod(r, tab->ql_mod[i], q);
        o[(long long)i * N + k] = add_mod(mul_shoup(cv[(long long)i * N + k], pinv[i], pinv_s[i], q), r, q);
    }
}

// out[b][t][i] = (x[b][t][i] - lifted[b][t][i]) * q_l^-1
__global__ void __launch_bounds__(kThreads) k_rescale_combine(const u64* __restrict__ x, int x_cap,
                                                              const u64* __restrict__ lifted, u64* __restrict__ out,
                                                              int out_cap, const RescaleTab* __restrict__ tab, int l,
                                                              int N) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y % l;
    const int bt = blockIdx.y / l;
    if (k >= N) return;
    const u64 q = tab->q[i];
    const u64 a = x[((long long)bt * x_cap + i) * N + k];
    const u64 c = lifted[((long long)bt * l + i) * N + k];
    out[((long long)bt * out_cap + i) * N + k] = mul_shoup(sub_mod(a, c, q), tab->qlinv[i], tab->qlinv_s[i], q);
}

// ---------------------------------------------------------------------------
// Tensor product of ciphertext pairs (evaluation form):
// d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1.  out: [B][3][level+1][N]
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_tensor(const TensorJobs jobs, int level,
                                                     const DevPrime* __restrict__ primes, int N) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    const TensorJob& J = jobs.j[blockIdx.z];
    if (k >= N) return;
    const DevPrime P = primes[i];
    const u64 a0 = J.a[(long long)i * N + k], a1 = J.a[((long long)J.a_cap + i) * N + k];
    const u64 b0 = J.b[(long long)i * N + k], b1 = J.b[((long long)J.b_cap + i) * N + k];
    const long long ps = (long long)(level + 1) * N;
    J.out[(long long)i * N + k] = mul_mod(a0, b0, P);
    J.out[ps + (long long)i * N + k] = add_mod(mul_mod(a0, b1, P), mul_mod(a1, b0, P), P.q);
    J.out[2 * ps + (long long)i * N + k] = mul_mod(a1, b1, P);
}

// ---------------------------------------------------------------------------
// Diagonal MAC (on-demand BSGS, Eq. eq:prerotation) for B queries at once:
//   P_{b,j}[t][i][k] = sum_{i' < n1, j n1 + i' < ell} baby_{b,i'}[t][i][k] * D'_{j n1 + i'}[i][k]
// A CTA owns TP evaluation points of one limb. The n1 baby words (both polys)
// of its points are staged in shared memory for every query; JG thread groups
// split the n2 giant steps. Every plaintext diagonal word is read once for all
// B queries, eight at a time per thread; when every batch of eight is full (n1 a
// multiple of 8 dividing ell), a word's register is refilled with the next batch's
// word as soon as it has been multiplied, so the loads stay in flight.
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(512, (B == 1 ? 2 : 1)) k_mac(const u64* __restrict__ babies, long long baby_q, int cap_b,
                                             const u64* __restrict__ diags, u64* __restrict__ out, long long out_q,
                                             int cap_o, int nl, int n1, int n2, int ell, int TP, int JG,
                                             const DevPrime* __restrict__ primes, int N) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ u64 sb[];  // [B][n1][2][TP]
    const int pl = threadIdx.x % TP;
    const int jg = threadIdx.x / TP;
    const int k = blockIdx.x * TP + pl;
    const int i = blockIdx.y;
    const u64 q = primes[i].q, qinv = primes[i].qinv, one_s = primes[i].one_s;
    const bool fold_each = n1 > 64;
    const int per_q = n1 * 2 * TP;
    // staging: thread (pl, jg) takes point pl of the rows r = 2 i' + t = jg, jg + JG, ... of
    // every query (no index divisions)
    {
        const long long rstep = (long long)cap_b * N;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const u64* src = babies + (long long)b * baby_q + (long long)i * N + k;
            u64* dst = sb + b * per_q + pl;
#pragma unroll 8
            for (int r = jg; r < 2 * n1; r += JG) dst[r * TP] = split30(src[r * rstep]);
        }
    }
    __syncthreads();
    const long long dstride = (long long)nl * N;
    // the thread's work is a sequence of batches (giant step j, 8 diagonals from i0)
    int j = jg, i0 = 0;
    if (j >= n2) return;
    const u64* sbase = sb + pl;
    const int TP2 = 2 * TP;
    Acc128 acc[B][2];
#pragma unroll
    for (int b = 0; b < B; ++b) acc[b][0] = acc[b][1] = Acc128{0, 0};
    // the products of one diagonal word d (both polys of every query's baby) into p
    auto mul_word = [&](AccK (&p)[B][2], u64 d, const u64* sq) {
        const u64 ds = split30(d);
        const u32 dsum = sum30(ds);
#pragma unroll
        for (int b = 0; b < B; ++b) {
            mack(p[b][0], ds, dsum, sq[b * per_q]);
            mack(p[b][1], ds, dsum, sq[b * per_q + TP]);
        }
    };
    // after a batch of giant step j: add its sums (a flush adds less than 2^60 to the high word,
    // so up to 64 products per giant step, 8 flushes, need no fold and the high word is reduced
    // once before the REDC); when the giant step ends, store it
    auto close_batch = [&](AccK (&p)[B][2], int jc, bool last) {
#pragma unroll
        for (int b = 0; b < B; ++b) {
            flushk(acc[b][0], p[b][0]);
            flushk(acc[b][1], p[b][1]);
            if (fold_each) {
                fold(acc[b][0], q);
                fold(acc[b][1], q);
            }
        }
        if (last) {
#pragma unroll
            for (int b = 0; b < B; ++b) {
                u64* O = out + (long long)b * out_q + (long long)jc * 2 * cap_o * N;
                O[(long long)i * N + k] = redc(mul_shoup(acc[b][0].hi, 1, one_s, q), acc[b][0].lo, q, qinv);
                O[((long long)cap_o + i) * N + k] = redc(mul_shoup(acc[b][1].hi, 1, one_s, q), acc[b][1].lo, q, qinv);
                acc[b][0] = acc[b][1] = Acc128{0, 0};
            }
        }
    };
    const u64* dbase = diags + (long long)i * N + k;
    if (ell % n1 == 0 && n1 % 8 == 0) {
        // every batch is full: while a batch is multiplied, each word's register is refilled with
        // the same word of the next batch, so eight loads per thread stay in flight throughout
        u64 d[8];
        {
            const u64* D = dbase + (long long)j * n1 * dstride;
#pragma unroll
            for (int u = 0; u < 8; ++u) d[u] = __ldcs(D + u * dstride);
        }
        for (;;) {
            int jn = j, in = i0 + 8;
            if (in == n1) {
                jn = j + JG;
                in = 0;
            }
            const bool more = jn < n2;
            const u64* Dn = dbase + ((long long)(more ? jn : j) * n1 + (more ? in : i0)) * dstride;
            const u64* s0 = sbase + i0 * TP2;
            AccK p[B][2];
#pragma unroll
            for (int b = 0; b < B; ++b) p[b][0] = p[b][1] = AccK{0, 0, 0};
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const u64 w = d[u];
                if (more) d[u] = __ldcs(Dn + u * dstride);
                mul_word(p, w, s0 + u * TP2);
            }
            close_batch(p, j, jn != j);
            if (!more) break;
            j = jn;
            i0 = in;
        }
        return;
    }
    for (;;) {
        const int cnt = min(n1, ell - j * n1);
        const u64* D = dbase + ((long long)j * n1 + i0) * dstride;
        const u64* s0 = sbase + i0 * TP2;
        AccK p[B][2];
#pragma unroll
        for (int b = 0; b < B; ++b) p[b][0] = p[b][1] = AccK{0, 0, 0};
        if (i0 + 8 <= cnt) {
            // full batch: no bounds checks
            u64 d[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) d[u] = __ldcs(D + u * dstride);
#pragma unroll
            for (int u = 0; u < 8; ++u) mul_word(p, d[u], s0 + u * TP2);
        } else {
            for (int u = 0; i0 + u < cnt; ++u) mul_word(p, __ldcs(D + (long long)u * dstride), s0 + u * TP2);
        }
        // next batch
        int jn = j, in = i0 + 8;
        if (in >= cnt) {
            jn = j + JG;
            in = 0;
        }
        close_batch(p, j, jn != j);
        if (jn >= n2) break;
        j = jn;
        i0 = in;
    }
}

// ---------------------------------------------------------------------------
// Diagonal MAC with the diagonals streamed through shared memory (the on-demand schedule's S4
// for B = 1..4 queries against one database, when n1 is a multiple of SD = 8 and n2 of JG): the
// sums of k_mac, P_{b,j}[t][i][k] = sum_{i'} B_{b,i'}[t][i][k] * D'_{j n1 + i'}[i][k], every
// diagonal word read once for all B queries. A CTA owns TP points of one limb and JG giant-step
// rows: thread (jg, point) accumulates giant steps jb JG + jg for its point. The babies of the
// CTA's points are staged once (30-bit halves, every query); the diagonals flow through a ring of
// kMpNS stages, stage (jb, i0) holding diagonals (jb JG + jg) n1 + i0 + u for jg < JG, u < SD,
// filled by 16-byte asynchronous copies (cp.async, one commit group per stage, kMpNS - 1 stages
// in flight while one is multiplied). A warp reads TP consecutive words of one row: no bank
// conflicts, and no exchange between threads until a giant step's sums are complete.
// ---------------------------------------------------------------------------
constexpr int kMpNS = 4;  // ring stages
constexpr int kMpSD = 8;  // diagonals of one giant step per stage (8 products between carries)

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory"); }

template <int B, int TP, int JG>
__global__ void __launch_bounds__(TP * JG) k_mac_pipe(const u64* __restrict__ babies, long long baby_q, int cap_b,
                                                      const u64* __restrict__ diags, u64* __restrict__ out,
                                                      long long out_q, int cap_o, int nl, int n1, int n2,
                                                      const DevPrime* __restrict__ primes, int N) {
    pdl_wait();
    pdl_trigger();
    constexpr int SD = kMpSD;
    constexpr int NT = TP * JG;                       // threads
    constexpr int ROWS = JG * SD;                     // diagonal rows per stage
    constexpr int CHUNKS = ROWS * TP / 2;             // 16-byte chunks per stage
    static_assert(CHUNKS % NT == 0, "whole chunks per thread");
    extern __shared__ __align__(16) u64 smp[];
    u64* sb = smp;                                    // babies [B][n1][2][TP], split
    u64* sd = sb + (size_t)B * n1 * 2 * TP;           // ring [NS][JG][SD][TP]
    const int i = blockIdx.y;
    const int k0 = blockIdx.x * TP;
    const int pl = threadIdx.x % TP, jg = threadIdx.x / TP;
    const u64 q = primes[i].q, qinv = primes[i].qinv;
    const int spb = n1 / SD;                          // stages per giant-step block
    const int nst = (n2 / JG) * spb;
    const int per_q = n1 * 2 * TP;
    auto issue = [&](int s) {
        if (s < nst) {
            const int jb = s / spb, i0 = (s % spb) * SD;
            u64* dst = sd + (size_t)(s % kMpNS) * ROWS * TP;
#pragma unroll
            for (int r = 0; r < CHUNKS / NT; ++r) {
                const int ch = threadIdx.x + r * NT;
                const int row = ch / (TP / 2), w = (ch % (TP / 2)) * 2;
                const int g = row / SD, u = row % SD;
                const long long d = (long long)(jb * JG + g) * n1 + i0 + u;
                cp_async16(dst + (size_t)row * TP + w, diags + (d * nl + i) * N + k0 + w);
            }
        }
        cp_async_commit();  // an empty group past the last stage keeps the group count uniform
    };
#pragma unroll
    for (int s = 0; s < kMpNS - 1; ++s) issue(s);
    for (int e = threadIdx.x; e < B * per_q; e += NT) {
        const int qb = e / per_q, r = e % per_q;
        const int ib = r / (2 * TP), t = (r / TP) & 1, pp = r % TP;
        sb[e] = split30(babies[(long long)qb * baby_q + ((long long)ib * 2 + t) * cap_b * N + (long long)i * N + k0 + pp]);
    }
    Acc128 acc[B][2];
#pragma unroll
    for (int qb = 0; qb < B; ++qb) acc[qb][0] = acc[qb][1] = Acc128{0, 0};
    for (int s = 0; s < nst; ++s) {
        cp_async_wait<kMpNS - 2>();  // this thread's copies of stage s have landed
        __syncthreads();             // every thread's have; slot (s - 1) % NS is free again
        issue(s + kMpNS - 1);
        const int jb = s / spb, i0 = (s % spb) * SD;
        const u64* st = sd + (size_t)(s % kMpNS) * ROWS * TP + (size_t)jg * SD * TP + pl;
        AccK p[B][2];
#pragma unroll
        for (int qb = 0; qb < B; ++qb) p[qb][0] = p[qb][1] = AccK{0, 0, 0};
#pragma unroll
        for (int u = 0; u < SD; ++u) {
            const u64 ds = split30(st[(size_t)u * TP]);
            const u32 dsum = sum30(ds);
#pragma unroll
            for (int qb = 0; qb < B; ++qb) {
                const u64* sq = sb + (size_t)qb * per_q + ((size_t)(i0 + u) * 2) * TP + pl;
                mack(p[qb][0], ds, dsum, sq[0]);
                mack(p[qb][1], ds, dsum, sq[TP]);
            }
        }
#pragma unroll
        for (int qb = 0; qb < B; ++qb) {
            flushk(acc[qb][0], p[qb][0]);
            flushk(acc[qb][1], p[qb][1]);
            fold(acc[qb][0], q);
            fold(acc[qb][1], q);
        }
        if (i0 + SD == n1) {
            // giant step jb JG + jg complete for this point: reduce and store
            const int j = jb * JG + jg;
#pragma unroll
            for (int qb = 0; qb < B; ++qb) {
                u64* O = out + (long long)qb * out_q + (long long)j * 2 * cap_o * N;
                O[(long long)i * N + k0 + pl] = redc(acc[qb][0].hi, acc[qb][0].lo, q, qinv);
                O[((long long)cap_o + i) * N + k0 + pl] = redc(acc[qb][1].hi, acc[qb][1].lo, q, qinv);
                acc[qb][0] = acc[qb][1] = Acc128{0, 0};
            }
        }
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Diagonal MAC as a persistent pipeline (the on-demand schedule's S4 for B = 1..4 queries against
// one database): the sums of k_mac, P_{b,j}[t][i][k] = sum_{i'} B_{b,i'}[t][i][k] D'_{j n1 + i'}[i][k].
// A tile is TP = 16 points of one limb; each CTA runs the tiles blockIdx.x, blockIdx.x + gridDim.x,
// ... with 256 threads, thread (giant-step row jg, point) accumulating giant steps jb 16 + jg. One
// ring of kMrNS stages of 16-byte asynchronous copies carries everything: stage (tile, jb, i0)
// holds diagonals (jb 16 + g) n1 + i0 + u, g < 16, u < 8, and the last stage of a tile also
// carries the next tile's babies (every query, raw residues) into the other of two baby buffers.
// So the copies of the next tile overlap the products of this one, and a CTA never waits for a
// tile's start. The babies of a tile are split into 30-bit halves in shared memory once, after
// they land. Every diagonal word is read once for all B queries. Needs n1 % 8 == 0, n2 % 16 == 0
// and at least kMrNS stages per tile (checked by mac_ring_fits).
// ---------------------------------------------------------------------------
constexpr int kMrNS = 3;   // ring stages
constexpr int kMrTP = 16;  // points per tile
constexpr int kMrJG = 16;  // giant-step rows per CTA

// Cursor over a CTA's stages (tile m, stage sl of the tile), advanced without divisions.
struct MrCursor {
    int m, sl, slot, tile, i, k0;
};

template <int B, int N1>
__global__ void __launch_bounds__(kMrTP * kMrJG) k_mac_ring(const u64* __restrict__ babies, long long baby_q,
                                                            int cap_b, const u64* __restrict__ diags,
                                                            u64* __restrict__ out, long long out_q, int cap_o, int nl,
                                                            int n2, const DevPrime* __restrict__ primes,
                                                            int N) {
    pdl_wait();
    pdl_trigger();
    constexpr int TP = kMrTP, JG = kMrJG, SD = kMpSD, NT = TP * JG, NS = kMrNS;
    constexpr int ROWS = JG * SD;          // diagonal rows per stage
    constexpr int CHUNKS = ROWS * TP / 2;  // 16-byte chunks per stage
    static_assert(CHUNKS % NT == 0, "whole chunks per thread");
    extern __shared__ __align__(16) u64 smr[];
    constexpr int qw = N1 * 2 * TP;        // words of one query's babies in a tile
    constexpr int bw = B * qw;             // words of one tile's babies
    u64* bb = smr;                         // [2][B][N1][2][TP]
    u64* sd = bb + 2 * (size_t)bw;         // ring [NS][JG][SD][TP]
    const int pl = threadIdx.x % TP, jg = threadIdx.x / TP;
    const int tpl = N / TP;                // tiles per limb
    const int ntile = nl * tpl;
    const int mt = (int)blockIdx.x < ntile ? (ntile - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    constexpr int spb = N1 / SD;           // stages per giant-step block
    const int nst = (n2 / JG) * spb;       // stages per tile
    const long long dstep = (long long)nl * N;  // one diagonal
    auto at_tile = [&](MrCursor& c) {
        c.tile = (int)blockIdx.x + c.m * (int)gridDim.x;
        c.i = c.tile / tpl;
        c.k0 = (c.tile - c.i * tpl) * TP;
    };
    auto advance = [&](MrCursor& c) {
        c.slot = c.slot + 1 == NS ? 0 : c.slot + 1;
        if (++c.sl == nst) {
            c.sl = 0;
            ++c.m;
            at_tile(c);
        }
    };
    auto issue = [&](const MrCursor& c) {
        if (c.m < mt) {
            const int jb = c.sl / spb, i0 = (c.sl - jb * spb) * SD;
            u64* dst = sd + (size_t)c.slot * ROWS * TP;
            const u64* src = diags + ((long long)jb * JG * N1 + i0) * dstep + (long long)c.i * N + c.k0;
#pragma unroll
            for (int r = 0; r < CHUNKS / NT; ++r) {
                const int ch = threadIdx.x + r * NT;
                const int row = ch / (TP / 2), w = (ch % (TP / 2)) * 2;
                const int gg = row / SD, u = row % SD;
                cp_async16(dst + (size_t)row * TP + w, src + ((long long)gg * N1 + u) * dstep + w);
            }
            // the babies of tile 0 ride on its first stage, those of tile m + 1 on tile m's last
            const int mb = (c.m == 0 && c.sl == 0) ? 0 : (c.sl == nst - 1 ? c.m + 1 : -1);
            if (mb >= 0 && mb < mt) {
                const int tb = (int)blockIdx.x + mb * (int)gridDim.x, il = tb / tpl, kb = (tb - il * tpl) * TP;
                u64* bd = bb + (size_t)(mb & 1) * bw;
                const u64* bs = babies + (long long)il * N + kb;
                for (int ch = threadIdx.x; ch < bw / 2; ch += NT) {
                    const int e = ch * 2;
                    const int qb = e / qw, r = e - qb * qw;
                    const int row = r / TP, pp = r - row * TP;  // row = 2 ib + t
                    cp_async16(bd + e, bs + (long long)qb * baby_q + (long long)row * cap_b * N + pp);
                }
            }
        }
        cp_async_commit();  // empty groups past the end keep the group count uniform
    };
    MrCursor ic{0, 0, 0, 0, 0, 0};  // issue cursor, NS - 1 stages ahead
    at_tile(ic);
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) {
        issue(ic);
        advance(ic);
    }
    MrCursor cc{0, 0, 0, 0, 0, 0};  // compute cursor
    at_tile(cc);
    Acc128 acc[B][2];
#pragma unroll
    for (int qb = 0; qb < B; ++qb) acc[qb][0] = acc[qb][1] = Acc128{0, 0};
    for (; cc.m < mt; advance(cc)) {
        cp_async_wait<NS - 2>();  // this thread's copies of this stage (and earlier) have landed
        __syncthreads();          // everyone's have; the ring slot before this one is free again
        issue(ic);
        advance(ic);
        u64* bm = bb + (size_t)(cc.m & 1) * bw;
        if (cc.sl == 0) {
            // a new tile: its babies have landed; split them into 30-bit halves in place
            for (int e = threadIdx.x; e < bw; e += NT) bm[e] = split30(bm[e]);
            __syncthreads();
        }
        const int jb = cc.sl / spb, i0 = (cc.sl - jb * spb) * SD;
        const u64* st = sd + (size_t)cc.slot * ROWS * TP + jg * SD * TP + pl;
        const u64* sq = bm + i0 * 2 * TP + pl;
        AccK p[B][2];
#pragma unroll
        for (int qb = 0; qb < B; ++qb) p[qb][0] = p[qb][1] = AccK{0, 0, 0};
#pragma unroll
        for (int u = 0; u < SD; ++u) {
            const u64 ds = split30(st[u * TP]);
            const u32 dsum = sum30(ds);
#pragma unroll
            for (int qb = 0; qb < B; ++qb) {
                mack(p[qb][0], ds, dsum, sq[qb * qw + u * 2 * TP]);
                mack(p[qb][1], ds, dsum, sq[qb * qw + u * 2 * TP + TP]);
            }
        }
        // no fold here: a flush adds less than 2^60 to the high word, and a giant step has at
        // most 8 flushes (N1 <= 64), so the high word is reduced once, before the REDC
#pragma unroll
        for (int qb = 0; qb < B; ++qb) {
            flushk(acc[qb][0], p[qb][0]);
            flushk(acc[qb][1], p[qb][1]);
        }
        if (i0 + SD == N1) {
            // giant step jb JG + jg complete for this point: reduce and store
            const DevPrime P = primes[cc.i];
            const int j = jb * JG + jg;
#pragma unroll
            for (int qb = 0; qb < B; ++qb) {
                u64* O = out + (long long)qb * out_q + (long long)j * 2 * cap_o * N + (long long)cc.i * N + cc.k0 + pl;
                O[0] = redc(mul_shoup(acc[qb][0].hi, 1, P.one_s, P.q), acc[qb][0].lo, P.q, P.qinv);
                O[(long long)cap_o * N] = redc(mul_shoup(acc[qb][1].hi, 1, P.one_s, P.q), acc[qb][1].lo, P.q, P.qinv);
                acc[qb][0] = acc[qb][1] = Acc128{0, 0};
            }
        }
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Encrypted-database MAC (ct x ct with lazy relinearisation, the paper's setting of
// Section 5.3): for every giant step j, pointwise per limb,
//   (d0, d1, d2)_j = sum_{i < n1, j n1 + i < ell} B_i (x) E_{j n1 + i}
//   d0 += b0 e0,  d1 += b0 e1 + b1 e0,  d2 += b1 e1.
// The middle term takes one product (Karatsuba): d1 = sum (b0 + b1)(e0 + e1) - d0 - d2, the
// same residue mod q as the two products it replaces.
// babies: [n1][2][cap_b][N] evaluation form; diags: [ell][2][nl][N] evaluation form in
// Montgomery form (e0 R + e1 R = (e0 + e1) R), so one REDC of each sum gives it in plain form;
// out: [n2][3][cap_o][N]. Tiling as k_mac: the babies of a point tile are staged in shared
// memory as 30-bit halves of b0, b1 and b0 + b1, giant steps run over the thread rows.
// Diagonals go in batches of 4 (one carry step per batch).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512, 2) k_mac_ct(const u64* __restrict__ babies, int cap_b,
                                                   const u64* __restrict__ diags, u64* __restrict__ out, int cap_o,
                                                   int nl, int n1, int n2, int ell, int TP, int JG,
                                                   const DevPrime* __restrict__ primes, int N) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ u64 sb[];  // [n1][3][TP]: b0, b1, b0 + b1
    const int pl = threadIdx.x % TP;
    const int jg = threadIdx.x / TP;
    const int k = blockIdx.x * TP + pl;
    const int i = blockIdx.y;
    const u64 q = primes[i].q, qinv = primes[i].qinv;
    // staging: thread (pl, jg) takes point pl of babies jg, jg + JG, ... (no index divisions)
#pragma unroll 4
    for (int ib = jg; ib < n1; ib += JG) {
        const u64* src = babies + (long long)ib * 2 * cap_b * N + (long long)i * N + k;
        const u64 b0 = src[0], b1 = src[(long long)cap_b * N];
        u64* dst = sb + (size_t)ib * 3 * TP + pl;
        dst[0] = split30(b0);
        dst[TP] = split30(b1);
        dst[2 * TP] = split30(add_mod(b0, b1, q));
    }
    __syncthreads();
    const long long dstride = 2LL * nl * N;  // one diagonal ciphertext
    const long long cstride = (long long)nl * N;
    for (int j = jg; j < n2; j += JG) {
        const int cnt = min(n1, ell - j * n1);
        const u64* D = diags + (long long)j * n1 * dstride + (long long)i * N + k;
        Acc128 a0{0, 0}, am{0, 0}, a2{0, 0};
        for (int i0 = 0; i0 < cnt; i0 += 4) {
            AccK p0{0, 0, 0}, pm{0, 0, 0}, p2{0, 0, 0};
            const u64* sq = sb + (size_t)i0 * 3 * TP + pl;
            if (i0 + 4 <= cnt) {
                u64 e0[4], e1[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    e0[u] = __ldcs(D + u * dstride);
                    e1[u] = __ldcs(D + u * dstride + cstride);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const u64* bq = sq + u * 3 * TP;
                    const u64 x0 = split30(e0[u]), x2 = split30(e1[u]), xm = split30(add_mod(e0[u], e1[u], q));
                    mack(p0, x0, sum30(x0), bq[0]);
                    mack(p2, x2, sum30(x2), bq[TP]);
                    mack(pm, xm, sum30(xm), bq[2 * TP]);
                }
            } else {
                for (int u = 0; i0 + u < cnt; ++u) {
                    const u64 f0 = __ldcs(D + u * dstride), f1 = __ldcs(D + u * dstride + cstride);
                    const u64* bq = sq + u * 3 * TP;
                    const u64 x0 = split30(f0), x2 = split30(f1), xm = split30(add_mod(f0, f1, q));
                    mack(p0, x0, sum30(x0), bq[0]);
                    mack(p2, x2, sum30(x2), bq[TP]);
                    mack(pm, xm, sum30(xm), bq[2 * TP]);
                }
            }
            flushk(a0, p0);
            flushk(am, pm);
            flushk(a2, p2);
            fold(a0, q);
            fold(am, q);
            fold(a2, q);
            D += 4 * dstride;
        }
        const u64 d0 = redc(a0.hi, a0.lo, q, qinv), d2 = redc(a2.hi, a2.lo, q, qinv);
        const u64 dm = redc(am.hi, am.lo, q, qinv);
        u64* O = out + (long long)j * 3 * cap_o * N + (long long)i * N + k;
        O[0] = d0;
        O[(long long)cap_o * N] = sub_mod(sub_mod(dm, d0, q), d2, q);
        O[2LL * cap_o * N] = d2;
    }
}

// ---------------------------------------------------------------------------
// Table-schedule MAC (Algorithm 1, step 4): S_g = sum_{m < ell} rotQ[m] (.) D_{g,m}
// for GG groups per CTA column. One thread per evaluation point of one limb; the two
// table words of a point are read once for the GG groups, the diagonal words streamed.
// table: [ell][2][cap_t][N]; diagonal m of group g, limb i at diags + g dgrp + (m nl + i) N
// (Montgomery form); output of group g at out + g og, [2][cap_o][N]. Products use the 30-bit
// split multiply-accumulate (four per carry step).
// ---------------------------------------------------------------------------
template <int GG>
__global__ void __launch_bounds__(256) k_mac_table(const u64* __restrict__ table, int cap_t,
                                                   const u64* __restrict__ diags, long long dgrp, int G,
                                                   u64* __restrict__ out, int cap_o, long long og, int nl, int ell,
                                                   const DevPrime* __restrict__ primes, int N) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    const int g0 = blockIdx.z * GG;
    if (k >= N) return;
    const u64 q = primes[i].q, qinv = primes[i].qinv;
    const long long ts = 2ll * cap_t * N, ds = (long long)nl * N;
    const u64* t0 = table + (long long)i * N + k;
    const u64* t1 = t0 + (long long)cap_t * N;
    const u64* d0 = diags + (long long)g0 * dgrp + (long long)i * N + k;
    Acc128 acc[GG][2];
#pragma unroll
    for (int gg = 0; gg < GG; ++gg) acc[gg][0] = acc[gg][1] = Acc128{0, 0};
    for (int m0 = 0; m0 < ell; m0 += 4) {
        u64 a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool ok = m0 + u < ell;
            a[u] = split30(ok ? t0[(long long)(m0 + u) * ts] : 0ull);
            b[u] = split30(ok ? t1[(long long)(m0 + u) * ts] : 0ull);
        }
#pragma unroll
        for (int gg = 0; gg < GG; ++gg) {
            if (g0 + gg < G) {
                AccK p0{0, 0, 0}, p1{0, 0, 0};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const u64 d = split30(m0 + u < ell ? __ldcs(d0 + gg * dgrp + (long long)(m0 + u) * ds) : 0ull);
                    const u32 dsum = sum30(d);
                    mack(p0, d, dsum, a[u]);
                    mack(p1, d, dsum, b[u]);
                }
                flushk(acc[gg][0], p0);
                flushk(acc[gg][1], p1);
                fold(acc[gg][0], q);
                fold(acc[gg][1], q);
            }
        }
    }
#pragma unroll
    for (int gg = 0; gg < GG; ++gg) {
        if (g0 + gg < G) {
            u64* O = out + (long long)(g0 + gg) * og;
            O[(long long)i * N + k] = redc(acc[gg][0].hi, acc[gg][0].lo, q, qinv);
            O[((long long)cap_o + i) * N + k] = redc(acc[gg][1].hi, acc[gg][1].lo, q, qinv);
        }
    }
}

// ---------------------------------------------------------------------------
// Elementwise helpers on ciphertext batches [B][2][cap][N] (evaluation form).
// ---------------------------------------------------------------------------
// out = a + b over limbs 0..level of both polys
__global__ void k_add(const u64* a, int a_cap, long long a_bs, const u64* b, int b_cap, long long b_bs, u64* out,
                      int o_cap, long long o_bs, int level, const DevPrime* primes, int N) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y % (level + 1);
    const int t = blockIdx.y / (level + 1);
    const int bb = blockIdx.z;
    if (k >= N) return;
    const u64 q = primes[i].q;
    const u64 x = a[bb * a_bs + ((long long)t * a_cap + i) * N + k];
    const u64 y = b[bb * b_bs + ((long long)t * b_cap + i) * N + k];
    out[bb * o_bs + ((long long)t * o_cap + i) * N + k] = add_mod(x, y, q);
}

// sum of J ciphertexts (stride js) into out
__global__ void k_sum(const u64* a, int cap, long long js, int J, u64* out, int o_cap, int level,
                      const DevPrime* primes, int N) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y % (level + 1);
    const int t = blockIdx.y / (level + 1);
    if (k >= N) return;
    const u64 q = primes[i].q;
    u64 v = 0;
    for (int j = 0; j < J; ++j) v = add_mod(v, a[j * js + ((long long)t * cap + i) * N + k], q);
    out[((long long)t * o_cap + i) * N + k] = v;
}

// Lifted last limbs of the Chebyshev leaves, T1 cb_j + ca_j at limb l, from u, the coefficient
// form of T1's last limb ([B][2][N]): the INTT is linear and the constant ca_j is the constant
// polynomial, so the leaf's last limb in coefficient form is cb_{j,l} u + ca_{j,l} at coefficient 0
// of component 0; centered and reduced to q_i for i < l as in k_rescale_lift.
// lifted [B nl][2][l][N]; grid (N / 256, 2 nl, B).
__global__ void k_leaf_lift(const u64* __restrict__ u, const u64* __restrict__ cb, const u64* __restrict__ cb_s,
                            const u64* __restrict__ ca, int nl, int L1, u64* __restrict__ lifted,
                            const RescaleTab* __restrict__ tab, u64 ql, int l, int N) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y >> 1, t = blockIdx.y & 1, b = blockIdx.z;
    if (k >= N) return;
    u64 r = mul_shoup(u[((long long)b * 2 + t) * N + k], cb[j * L1 + l], cb_s[j * L1 + l], ql);
    if (t == 0 && k == 0) r = add_mod(r, ca[j * L1 + l], ql);
    const bool neg = r > tab->half;
    u64* o = lifted + ((((long long)b * nl + j) * 2 + t) * l) * N + k;
    for (int i = 0; i < l; ++i) {
        const u64 q = tab->q[i];
        u64 w = mul_shoup(r, 1, tab->one_s[i], q);
        if (neg) w = sub_mod(w, tab->ql_mod[i], q);
        o[(long long)i * N] = w;
    }
}

// x <- 2 x - c (c added to the constant term: every evaluation point of c0)
__global__ void k_to_mont(u64* x, long long n_per_poly, PrimeMap pm, const DevPrime* primes, long long total) {
    pdl_wait();
    pdl_trigger();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(e / n_per_poly);
        const DevPrime P = primes[pm.idx[p % pm.period]];
        x[e] = to_mont(x[e], P);
    }
}

// ---------------------------------------------------------------------------
// Device slot encoder for template diagonals (reading R5, same operations and
// order as the host encoder: inverse special FFT stages len = n..2, bit
// reversal, times 1/n and Delta, rounded half away from zero).
// Stage arithmetic uses explicitly rounded intrinsics (no contraction).
// ---------------------------------------------------------------------------
struct cplx {
    double r, i;
};

__device__ __forceinline__ void fft_inv_bfly(cplx& a, cplx& b, double wr, double wi) {
    const double sr = __dadd_rn(a.r, b.r), si = __dadd_rn(a.i, b.i);
    const double dr = __dsub_rn(a.r, b.r), di = __dsub_rn(a.i, b.i);
    a.r = sr;
    a.i = si;
    b.r = __dsub_rn(__dmul_rn(dr, wr), __dmul_rn(di, wi));
    b.i = __dadd_rn(__dmul_rn(dr, wi), __dmul_rn(di, wr));
}

// Gather of the pre-rotated diagonals into slot vectors:
// z[x] = diag_d(M_k)[(x - shift) mod n], diag_d(M_k)[b ell + r] = T[(k B + b) ell + r][(r + d) mod ell]
__global__ void k_diag_gather(const float* __restrict__ T, long long K, int ell, int n, long long grp, int d0, int nd,
                              int n1, cplx* __restrict__ z) {
    pdl_wait();
    pdl_trigger();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int di = blockIdx.y;
    if (x >= n || di >= nd) return;
    const int d = d0 + di;
    const long long shift = (long long)(d / n1) * n1;
    long long y = ((long long)x - shift) % n;
    if (y < 0) y += n;
    const long long B = n / ell;
    const long long b = y / ell, r = y % ell;
    const long long row = (grp * B + b) * ell + r;
    const double v = row < K ? (double)T[row * ell + (r + d) % ell] : 0.0;
    z[(long long)di * n + x] = cplx{v, 0.0};
}

// first log2(R) stages (len = n .. 2n/R): columns of stride n/R; one tile of 16 columns
__global__ void __launch_bounds__(256) k_fft_col(cplx* z, int logn, int logR, const unsigned* rot, const double* zr,
                                                 const double* zi) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ cplx sc[];
    const int n = 1 << logn, Rr = 1 << logR, C = n >> logR;
    const int TC = 16;
    const long long M = 4ll * n;
    cplx* x = z + (long long)blockIdx.y * n;
    const int col0 = blockIdx.x * TC;
    for (int e = threadIdx.x; e < Rr * TC; e += blockDim.x) {
        int r = e / TC, c = e % TC;
        sc[e] = x[(long long)r * C + col0 + c];
    }
    __syncthreads();
    for (int len = n; len >= 2 * C; len >>= 1) {
        const int hrow = (len >> 1) / C;  // half block in rows
        const long long lq = (long long)len << 2, gap = M / lq;  // powers of two
        for (int bf = threadIdx.x; bf < (Rr >> 1) * TC; bf += blockDim.x) {
            int c = bf % TC, pr = bf / TC;
            int blk = pr / hrow, u = pr - blk * hrow;
            int ra = blk * 2 * hrow + u, rb = ra + hrow;
            const int j = (col0 + c) + u * C;  // position inside the len-block
            const long long idx = (lq - (long long)(rot[j] & (unsigned)(lq - 1))) * gap;
            fft_inv_bfly(sc[ra * TC + c], sc[rb * TC + c], zr[idx], zi[idx]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < Rr * TC; e += blockDim.x) {
        int r = e / TC, c = e % TC;
        x[(long long)r * C + col0 + c] = sc[e];
    }
}

// remaining stages (len = C .. 2) inside contiguous blocks of C
__global__ void __launch_bounds__(256) k_fft_row(cplx* z, int logn, int logR, int bpc, const unsigned* rot,
                                                 const double* zr, const double* zi) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ cplx sc[];
    const int n = 1 << logn, C = n >> logR;
    const long long M = 4ll * n;
    cplx* x = z + (long long)blockIdx.y * n + (long long)blockIdx.x * bpc * C;
    const int tile = bpc * C;
    for (int e = threadIdx.x; e < tile; e += blockDim.x) sc[e] = x[e];
    __syncthreads();
    for (int len = C; len >= 2; len >>= 1) {
        const int h = len >> 1;
        const long long lq = (long long)len << 2, gap = M / lq;
        for (int bf = threadIdx.x; bf < tile / 2; bf += blockDim.x) {
            int blk = bf / h, u = bf - blk * h;
            int a = blk * len + u, b = a + h;
            const long long idx = (lq - (long long)(rot[u] & (unsigned)(lq - 1))) * gap;
            fft_inv_bfly(sc[a], sc[b], zr[idx], zi[idx]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < tile; e += blockDim.x) x[e] = sc[e];
}

// coefficient c of the encoded diagonal di: bit reversal, times 1/n and Delta, rounded half
// away from zero
__device__ __forceinline__ long long fft_coef(const cplx* __restrict__ z, int logn, int di, int c, int scale_bits) {
    const int n = 1 << logn;
    const int cc = c < n ? c : c - n;
    const int src = __brev(cc) >> (32 - logn);
    const cplx w = z[(long long)di * n + src];
    const double v = c < n ? w.r : w.i;
    const double inv_n = 1.0 / (double)n;
    const double delta = ldexp(1.0, scale_bits);
    return llround(__dmul_rn(__dmul_rn(v, inv_n), delta));
}

// m mod q for a signed coefficient: |m| reduced with the Shoup quotient of 1
__device__ __forceinline__ u64 coef_residue(long long m, const DevPrime& P) {
    const bool neg = m < 0;
    const u64 a = neg ? (u64)(-(m + 1)) : (u64)m;
    const u64 ra = mul_shoup(a, 1, P.one_s, P.q);
    return neg ? P.q - 1 - ra : ra;
}

// rounding and residues: out [nd][nl][N] (coefficient form)
__global__ void k_fft_finish(const cplx* __restrict__ z, int logn, int nd, u64* __restrict__ out, int nl,
                             const DevPrime* __restrict__ primes, int scale_bits) {
    pdl_wait();
    pdl_trigger();
    const int N = 2 << logn;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int di = blockIdx.y;
    if (c >= N || di >= nd) return;
    const long long m = fft_coef(z, logn, di, c, scale_bits);
    u64* o = out + (long long)di * nl * N;
    for (int i = 0; i < nl; ++i) o[(long long)i * N + c] = coef_residue(m, primes[i]);
}

// rounding only: the integer coefficients m [nd][N] (storage tier B)
__global__ void k_fft_round(const cplx* __restrict__ z, int logn, int nd, long long* __restrict__ out,
                            int scale_bits) {
    pdl_wait();
    pdl_trigger();
    const int N = 2 << logn;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int di = blockIdx.y;
    if (c >= N || di >= nd) return;
    out[(long long)di * N + c] = fft_coef(z, logn, di, c, scale_bits);
}

// residues of stored integer coefficients: m [nd][N] -> out [nd][nl][N]
__global__ void k_coef_residues(const long long* __restrict__ m, int nd, u64* __restrict__ out, int nl,
                                const DevPrime* __restrict__ primes, int N) {
    pdl_wait();
    pdl_trigger();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int di = blockIdx.y;
    if (c >= N || di >= nd) return;
    const long long v = m[(long long)di * N + c];
    u64* o = out + (long long)di * nl * N;
    for (int i = 0; i < nl; ++i) o[(long long)i * N + c] = coef_residue(v, primes[i]);
}

}  // namespace

// ===========================================================================
// launchers
// ===========================================================================

void launch_modup(const u64* in, long long in_job, const u64* in_eval, long long eval_job, u64* ext,
                  const ModUpTab* tabs, int beta, int npos, int N, int J, cudaStream_t s) {
    dim3 g((N + kThreads - 1) / kThreads, beta, J);
    launch_k(k_modup, dim3(g), dim3(kThreads), 0, s, in, in_job, in_eval, eval_job, ext, tabs, beta, npos, N);
}

void launch_ip(const IPJobs& jobs, int beta, int npos, int level, int kp, int T, const DevPrime* primes,
               const PrimeMap& pos_prime, int logN, cudaStream_t s, const u64* pmod, const u64* pmod_s) {
    const int N = 1 << logN;
    dim3 g((N + kThreads - 1) / kThreads, jobs.ngroups, npos);
    const int pbase = npos > level + 1 ? pos_prime.idx[level + 1] : 0;
    switch (beta) {
#define FR_IP_CASE(B) \
    case B: launch_k(k_ip<B>, g, dim3(kThreads), 0, s, jobs, npos, level, kp, T, primes, pbase, logN, pmod, pmod_s); \
        break;
        FR_IP_CASE(1) FR_IP_CASE(2) FR_IP_CASE(3) FR_IP_CASE(4) FR_IP_CASE(5) FR_IP_CASE(6) FR_IP_CASE(7)
        default: launch_k(k_ip<8>, g, dim3(kThreads), 0, s, jobs, npos, level, kp, T, primes, pbase, logN, pmod, pmod_s);
            break;
#undef FR_IP_CASE
    }
}

void launch_ip_sum(const IPSumJobs& jobs, int beta, int npos, int level, int kp, int T, const DevPrime* primes,
                   const PrimeMap& pos_prime, int logN, const u64* pmod, const u64* pmod_s, cudaStream_t s) {
    const int N = 1 << logN;
    dim3 g((N + kThreads - 1) / kThreads, jobs.ngroups, npos);
    const int pbase = npos > level + 1 ? pos_prime.idx[level + 1] : 0;
    switch (beta) {
#define FR_IPS_CASE(B) \
    case B: launch_k(k_ip_sum<B>, g, dim3(kThreads), 0, s, jobs, npos, level, kp, T, primes, pbase, logN, pmod, pmod_s); \
        break;
        FR_IPS_CASE(1) FR_IPS_CASE(2) FR_IPS_CASE(3) FR_IPS_CASE(4) FR_IPS_CASE(5) FR_IPS_CASE(6) FR_IPS_CASE(7)
        default: launch_k(k_ip_sum<8>, g, dim3(kThreads), 0, s, jobs, npos, level, kp, T, primes, pbase, logN, pmod,
                          pmod_s);
            break;
#undef FR_IPS_CASE
    }
}

void launch_p2q(const u64* acc, long long acc_job, int npos, int level, u64* conv, const P2QTab* tab, int N, int J,
                cudaStream_t s) {
    dim3 g((N + kThreads - 1) / kThreads, 2, J);
    launch_k(k_p2q, dim3(g), dim3(kThreads), 0, s, acc, acc_job, npos, level, conv, tab, N);
}

void launch_moddown_combine(const MDJobs& jobs, int J, int npos, int level, const u64* pinv, const u64* pinv_s,
                            const DevPrime* primes, int logN, cudaStream_t s) {
    const int N = 1 << logN;
    dim3 g((N + kThreads - 1) / kThreads, 2 * (level + 1), J);
    launch_k(k_moddown_combine, dim3(g), dim3(kThreads), 0, s, jobs, npos, level, pinv, pinv_s, primes, logN);
}

void launch_baby0_pq(u64* babies, long long baby_q, const u64* q, long long q_bs, int q_cap, int B, int npos,
                     int level, const DevPrime* primes, const u64* pmod, const u64* pmod_s, int N, cudaStream_t s) {
    dim3 g((N + kThreads - 1) / kThreads, npos, 2 * B);
    launch_k(k_baby0_pq, g, dim3(kThreads), 0, s, babies, baby_q, q, q_bs, q_cap, npos, level, primes, pmod, pmod_s, N);
}

void launch_rs_last(const u64* acc, const u64* d, u64* z, const u64* pinv, const u64* pinv_s, int npos, int l,
                    const DevPrime* primes, int N, int J, cudaStream_t s) {
    dim3 g((N + kThreads - 1) / kThreads, 2 * J);
    launch_k(k_rs_last, g, dim3(kThreads), 0, s, acc, d, z, pinv, pinv_s, npos, l, primes, N);
}

void launch_rs_lift(const u64* zc, const u64* conv, u64* y, const u64* pinv, const u64* pinv_s, const RescaleTab* tab,
                    const DevPrime* primes, int l, int N, int J, cudaStream_t s) {
    dim3 g((N + kThreads - 1) / kThreads, 2 * J);
    launch_k(k_rs_lift, g, dim3(kThreads), 0, s, zc, conv, y, pinv, pinv_s, tab, primes, l, N);
}

void launch_rescale_lift(const u64* last, u64* lifted, const RescaleTab* tab, int l, int N, int BT, cudaStream_t s) {
    dim3 g((N + kThreads - 1) / kThreads, BT);
    launch_k(k_rescale_lift, dim3(g), dim3(kThreads), 0, s, last, lifted, tab, l, N);
}

void launch_rescale_combine(const u64* x, int x_cap, const u64* lifted, u64* out, int out_cap, const RescaleTab* tab,
                            int l, int N, int BT, cudaStream_t s) {
    dim3 g((N + kThreads - 1) / kThreads, BT * l);
    launch_k(k_rescale_combine, dim3(g), dim3(kThreads), 0, s, x, x_cap, lifted, out, out_cap, tab, l, N);
}

void launch_tensor(const TensorJobs& jobs, int J, int level, const DevPrime* primes, int N, cudaStream_t s) {
    dim3 g((N + kThreads - 1) / kThreads, level + 1, J);
    launch_k(k_tensor, dim3(g), dim3(kThreads), 0, s, jobs, level, primes, N);
}

template <int B>
static void launch_mac_t(const u64* babies, long long baby_q, int cap_b, const u64* diags, u64* out, long long out_q,
                         int cap_o, int nl, int n1, int n2, int ell, const DevPrime* primes, int N, cudaStream_t s) {
    // points per CTA: staged babies (B n1 2 TP words) within 128 KiB; giant-step groups up to 512 threads
    int TP = 128;
    while (TP > 16 && (size_t)B * n1 * 2 * TP * 8 > (128u << 10)) TP >>= 1;
    int JG = 512 / TP;
    if (JG > n2) JG = n2;
    if (JG < 1) JG = 1;
    const size_t sm = (size_t)B * n1 * 2 * TP * sizeof(u64);
    static std::atomic<unsigned long long> attr{0};
    smem_limit_once(k_mac<B>, 200 * 1024, attr);
    dim3 g(N / TP, nl);
    launch_k(k_mac<B>, dim3(g), dim3(TP * JG), sm, s, babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, ell, TP, JG, primes, N);
}

static size_t mac_ring_smem(int B, int n1) {
    return ((size_t)2 * B * n1 * 2 * kMrTP + (size_t)kMrNS * kMrJG * kMpSD * kMrTP) * sizeof(u64);
}

bool mac_ring_fits(int n1, int ell, int N, int B) {
    // instantiated for n1 = 32 (the headline BSGS split); other splits take k_mac_pipe or k_mac
    if (n1 != 32 || ell % n1 != 0 || N % kMrTP != 0 || B < 1 || B > 4) return false;
    const int n2 = ell / n1;
    if (n1 > 64 || n2 % kMrJG != 0 || (n2 / kMrJG) * (n1 / kMpSD) < kMrNS) return false;
    return mac_ring_smem(B, n1) <= 200u * 1024;
}

template <int B>
static void launch_mac_ring_t(const u64* babies, long long baby_q, int cap_b, const u64* diags, u64* out,
                              long long out_q, int cap_o, int nl, int n1, int n2, const DevPrime* primes, int N,
                              cudaStream_t s) {
    const size_t sm = mac_ring_smem(B, n1);
    static std::atomic<unsigned long long> attr{0};
    smem_limit_once(k_mac_ring<B, 32>, 200 * 1024, attr);
    // persistent grid: as many CTAs as fit on the GPU at once, capped by the tile count
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mac_ring<B, 32>, kMrTP * kMrJG, sm);
    const long long ntile = (long long)nl * (N / kMrTP);
    const int grid = (int)std::min<long long>(ntile, (long long)std::max(1, per) * std::max(1, sms));
    launch_k(k_mac_ring<B, 32>, dim3(grid), dim3(kMrTP * kMrJG), sm, s, babies, baby_q, cap_b, diags, out, out_q,
             cap_o, nl, n2, primes, N);
}

void launch_mac_ring(const u64* babies, long long baby_q, int cap_b, const u64* diags, u64* out, long long out_q,
                     int cap_o, int nl, int n1, int ell, int B, const DevPrime* primes, int N, cudaStream_t s) {
    const int n2 = ell / n1;
    switch (B) {
        case 1: launch_mac_ring_t<1>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, primes, N, s); break;
        case 2: launch_mac_ring_t<2>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, primes, N, s); break;
        case 3: launch_mac_ring_t<3>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, primes, N, s); break;
        case 4: launch_mac_ring_t<4>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, primes, N, s); break;
        default: break;  // the engine splits larger batches
    }
}

bool mac_pipe_fits(int n1, int ell, int N) {
    const int n2 = n1 > 0 ? ell / n1 : 0;
    return n1 % kMpSD == 0 && n1 <= 64 && ell % n1 == 0 && n2 % 4 == 0 && N % 64 == 0;
}

// TP points x JG giant-step rows per CTA. One query: 64 points x 4 rows. Two to four queries:
// 16 points x 16 rows when the giant steps come in blocks of 16 (256 threads; 8 B KiB of staged
// babies and a 64 KiB ring, so two CTAs, 16 warps, share an SM), else 32 points x 4 rows.
template <int B, int TP, int JG>
static void launch_mac_pipe_s(const u64* babies, long long baby_q, int cap_b, const u64* diags, u64* out,
                              long long out_q, int cap_o, int nl, int n1, int n2, const DevPrime* primes, int N,
                              cudaStream_t s) {
    const size_t sm = ((size_t)B * n1 * 2 * TP + (size_t)kMpNS * JG * kMpSD * TP) * sizeof(u64);
    // the limit is raised once per device, so to the most any n1 <= 64 needs (200 KiB)
    static std::atomic<unsigned long long> attr{0};
    smem_limit_once(k_mac_pipe<B, TP, JG>, 200 * 1024, attr);
    dim3 g(N / TP, nl);
    launch_k(k_mac_pipe<B, TP, JG>, g, dim3(TP * JG), sm, s, babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1,
             n2, primes, N);
}

template <int B>
static void launch_mac_pipe_t(const u64* babies, long long baby_q, int cap_b, const u64* diags, u64* out,
                              long long out_q, int cap_o, int nl, int n1, int n2, const DevPrime* primes, int N,
                              cudaStream_t s) {
    if constexpr (B == 1) {
        launch_mac_pipe_s<1, 64, 4>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, primes, N, s);
    } else {
        if (n2 % 16 == 0 && N % 16 == 0)
            launch_mac_pipe_s<B, 16, 16>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, primes, N, s);
        else
            launch_mac_pipe_s<B, 32, 4>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, primes, N, s);
    }
}

void launch_mac_pipe(const u64* babies, long long baby_q, int cap_b, const u64* diags, u64* out, long long out_q,
                     int cap_o, int nl, int n1, int ell, int B, const DevPrime* primes, int N, cudaStream_t s) {
    const int n2 = ell / n1;
    switch (B) {
        case 1: launch_mac_pipe_t<1>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, primes, N, s); break;
        case 2: launch_mac_pipe_t<2>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, primes, N, s); break;
        case 3: launch_mac_pipe_t<3>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, primes, N, s); break;
        case 4: launch_mac_pipe_t<4>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, primes, N, s); break;
        default: break;  // the engine splits larger batches
    }
}

void launch_mac(const u64* babies, long long baby_q, int cap_b, const u64* diags, u64* out, long long out_q,
                int cap_o, int nl, int n1, int n2, int ell, int B, const DevPrime* primes, int N, cudaStream_t s) {
    switch (B) {
        case 1: launch_mac_t<1>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, ell, primes, N, s); break;
        case 2: launch_mac_t<2>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, ell, primes, N, s); break;
        case 3: launch_mac_t<3>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, ell, primes, N, s); break;
        case 4: launch_mac_t<4>(babies, baby_q, cap_b, diags, out, out_q, cap_o, nl, n1, n2, ell, primes, N, s); break;
        default: break;  // the engine splits larger batches
    }
}

void launch_mac_ct(const u64* babies, int cap_b, const u64* diags, u64* out, int cap_o, int nl, int n1, int n2, int ell,
                   const DevPrime* primes, int N, cudaStream_t s) {
    // points per CTA: staged babies (n1 3 TP words) within 128 KiB; giant-step rows up to 512 threads
    int TP = 128;
    while (TP > 16 && (size_t)n1 * 3 * TP * 8 > (128u << 10)) TP >>= 1;
    int JG = 512 / TP;
    if (JG > n2) JG = n2;
    if (JG < 1) JG = 1;
    const size_t sm = (size_t)n1 * 3 * TP * sizeof(u64);
    static std::atomic<unsigned long long> attr{0};
    smem_limit_once(k_mac_ct, 200 * 1024, attr);
    dim3 g(N / TP, nl);
    launch_k(k_mac_ct, dim3(g), dim3(TP * JG), sm, s, babies, cap_b, diags, out, cap_o, nl, n1, n2, ell, TP, JG, primes, N);
}

void launch_mac_table(const u64* table, int cap_t, const u64* diags, long long dgrp, int G, u64* out, int cap_o,
                      long long og, int nl, int ell, const DevPrime* primes, int N, cudaStream_t s) {
    const int GG = G >= 8 ? 8 : G >= 4 ? 4 : G >= 2 ? 2 : 1;
    dim3 g((N + kThreads - 1) / kThreads, nl, (G + GG - 1) / GG);
    switch (GG) {
        case 8: launch_k(k_mac_table<8>, dim3(g), dim3(kThreads), 0, s, table, cap_t, diags, dgrp, G, out, cap_o, og, nl, ell, primes, N); break;
        case 4: launch_k(k_mac_table<4>, dim3(g), dim3(kThreads), 0, s, table, cap_t, diags, dgrp, G, out, cap_o, og, nl, ell, primes, N); break;
        case 2: launch_k(k_mac_table<2>, dim3(g), dim3(kThreads), 0, s, table, cap_t, diags, dgrp, G, out, cap_o, og, nl, ell, primes, N); break;
        default: launch_k(k_mac_table<1>, dim3(g), dim3(kThreads), 0, s, table, cap_t, diags, dgrp, G, out, cap_o, og, nl, ell, primes, N); break;
    }
}

void launch_add(const u64* a, int a_cap, long long a_bs, const u64* b, int b_cap, long long b_bs, u64* out, int o_cap,
                long long o_bs, int level, int B, const DevPrime* primes, int N, cudaStream_t s) {
    dim3 g((N + kThreads - 1) / kThreads, 2 * (level + 1), B);
    launch_k(k_add, dim3(g), dim3(kThreads), 0, s, a, a_cap, a_bs, b, b_cap, b_bs, out, o_cap, o_bs, level, primes, N);
}

void launch_sum(const u64* a, int cap, long long js, int J, u64* out, int o_cap, int level, const DevPrime* primes,
                int N, cudaStream_t s) {
    dim3 g((N + kThreads - 1) / kThreads, 2 * (level + 1));
    launch_k(k_sum, dim3(g), dim3(kThreads), 0, s, a, cap, js, J, out, o_cap, level, primes, N);
}

void launch_leaf_lift(const u64* u, const u64* cb, const u64* cb_s, const u64* ca, int nl, int L1, u64* lifted,
                      const RescaleTab* tab, u64 ql, int l, int N, int B, cudaStream_t s) {
    dim3 g((N + kThreads - 1) / kThreads, 2 * nl, B);
    launch_k(k_leaf_lift, dim3(g), dim3(kThreads), 0, s, u, cb, cb_s, ca, nl, L1, lifted, tab, ql, l, N);
}

void launch_to_mont(u64* x, long long n_per_poly, const PrimeMap& pm, const DevPrime* primes, long long total,
                    cudaStream_t s) {
    long long blocks = (total + kThreads - 1) / kThreads;
    if (blocks > 152 * 32) blocks = 152 * 32;
    launch_k(k_to_mont, dim3((unsigned)blocks), dim3(kThreads), 0, s, x, n_per_poly, pm, primes, total);
}

static void encode_fft(const float* T, long long K, int ell, int logn, long long grp, int d0, int nd, int n1,
                       cplx* z, const unsigned* rot, const double* zr, const double* zi, cudaStream_t s) {
    const int n = 1 << logn;
    {
        dim3 g((n + kThreads - 1) / kThreads, nd);
        launch_k(k_diag_gather, dim3(g), dim3(kThreads), 0, s, T, K, ell, n, grp, d0, nd, n1, z);
    }
    const int logR = logn / 2;
    const int Rr = 1 << logR, C = n >> logR;
    {
        dim3 g(C / 16, nd);
        const size_t sm = (size_t)Rr * 16 * sizeof(cplx);
        launch_k(k_fft_col, dim3(g), dim3(256), sm, s, z, logn, logR, rot, zr, zi);
    }
    {
        int bpc = 1024 / C;
        if (bpc < 1) bpc = 1;
        if (bpc > Rr) bpc = Rr;
        dim3 g(Rr / bpc, nd);
        const size_t sm = (size_t)bpc * C * sizeof(cplx);
        launch_k(k_fft_row, dim3(g), dim3(256), sm, s, z, logn, logR, bpc, rot, zr, zi);
    }
}

void launch_encode_diags(const float* T, long long K, int ell, int logn, long long grp, int d0, int nd, int n1,
                         void* zbuf, u64* out_coeff, int nl, const DevPrime* primes, int scale_bits,
                         const unsigned* rot, const double* zr, const double* zi, cudaStream_t s) {
    const int n = 1 << logn;
    cplx* z = (cplx*)zbuf;
    encode_fft(T, K, ell, logn, grp, d0, nd, n1, z, rot, zr, zi, s);
    dim3 g((2 * n + kThreads - 1) / kThreads, nd);
    launch_k(k_fft_finish, dim3(g), dim3(kThreads), 0, s, z, logn, nd, out_coeff, nl, primes, scale_bits);
}

void launch_encode_diags_int(const float* T, long long K, int ell, int logn, long long grp, int d0, int nd, int n1,
                             void* zbuf, long long* out_int, int scale_bits, const unsigned* rot, const double* zr,
                             const double* zi, cudaStream_t s) {
    const int n = 1 << logn;
    cplx* z = (cplx*)zbuf;
    encode_fft(T, K, ell, logn, grp, d0, nd, n1, z, rot, zr, zi, s);
    dim3 g((2 * n + kThreads - 1) / kThreads, nd);
    launch_k(k_fft_round, dim3(g), dim3(kThreads), 0, s, z, logn, nd, out_int, scale_bits);
}

void launch_coef_residues(const long long* m, int nd, u64* out, int nl, const DevPrime* primes, int N,
                          cudaStream_t s) {
    dim3 g((N + kThreads - 1) / kThreads, nd);
    launch_k(k_coef_residues, dim3(g), dim3(kThreads), 0, s, m, nd, out, nl, primes, N);
}

namespace {

// Register-only FP64 fused multiply-add throughput (the ceiling of the encoder's FFT): eight
// independent chains per thread, x <- x a + b, with a slightly below 1 so values stay finite.
__global__ void __launch_bounds__(256) k_fp64_peak(double a, double b, int iters, double* sink) {
    double x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = 1.0 + 1e-3 * (threadIdx.x * 8 + e);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = __fma_rn(x[e], a, b);
    }
    double acc = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) acc += x[e];
    if (acc == -1.0) sink[0] = acc;  // keeps the loop live
}

}  // namespace

double measure_fp64_peak(int device) {
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    double* sink = nullptr;
    if (cudaMalloc(&sink, 8) != cudaSuccess) return 0;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_fp64_peak<<<blocks, threads>>>(0.999999, 1e-9, 64, sink);  // warm-up
    cudaEventRecord(a);
    k_fp64_peak<<<blocks, threads>>>(0.999999, 1e-9, iters, sink);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    if (ms <= 0) return 0;
    return 2.0 * blocks * threads * 8.0 * iters / (ms * 1e-3);  // an FMA is two operations
}
