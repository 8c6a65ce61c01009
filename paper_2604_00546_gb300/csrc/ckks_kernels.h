// Tables and launchers of the CKKS device kernels.
#pragma once
#include "kernels.h"

#define FR_MAX_DIGIT_LIMBS 16

// ModUp constants of one digit at one level: sources are the digit's Q limbs
// [lo, lo + ns); targets are every position of Q_l u P.
// FastBConv constants. hat_m holds [B/b_i]_t in Montgomery form (times 2^64 mod t), split into
// 30-bit halves (low half in bits 0..29, high half in bits 32..61) for the multiply-accumulate;
// tinv = t^-1 mod 2^64 and t_one_s = floor(2^64 / t) reduce the sum.
struct ModUpTab {
    int ns, lo;
    u64 src_q[FR_MAX_DIGIT_LIMBS];
    u64 inv_hat[FR_MAX_DIGIT_LIMBS], inv_hat_s[FR_MAX_DIGIT_LIMBS];
    u64 tq[FR_MAX_PRIMES];
    u64 tinv[FR_MAX_PRIMES], t_one_s[FR_MAX_PRIMES];
    u64 hat_m[FR_MAX_DIGIT_LIMBS][FR_MAX_PRIMES];
};

// ModDown constants: sources are the P limbs, targets Q limbs 0..l
struct P2QTab {
    int np;
    u64 pq[FR_MAX_DIGIT_LIMBS];
    u64 inv_hat[FR_MAX_DIGIT_LIMBS], inv_hat_s[FR_MAX_DIGIT_LIMBS];
    u64 qq[FR_MAX_PRIMES];
    u64 qinv[FR_MAX_PRIMES], q_one_s[FR_MAX_PRIMES];
    u64 hat_m[FR_MAX_DIGIT_LIMBS][FR_MAX_PRIMES];
};

// Rescale constants at level l (divide by q_l)
struct RescaleTab {
    u64 half;  // (q_l - 1) / 2
    u64 q[FR_MAX_PRIMES];
    u64 one_s[FR_MAX_PRIMES];  // floor(2^64 / q_i): Shoup quotient of 1, for x mod q_i
    u64 ql_mod[FR_MAX_PRIMES];
    u64 qlinv[FR_MAX_PRIMES], qlinv_s[FR_MAX_PRIMES];
};

struct IPJob {
    const u64* ext;  // [beta][npos][N]
    const u64* key;  // [digits][2][T][N], Montgomery form: Q limbs 0..kp-1, then P limbs
    u64* out;        // [2][npos][N]
    u32 galois;      // 1: no automorphism
    u32 pad;
    const u64* addb = nullptr;  // non-null: add P sigma_galois(addb) to component 0 on the Q positions
                                // (addb: limbs 0..level, stride N, evaluation form)
};

struct MDJob {
    const u64* acc;   // [2][npos][N]
    const u64* conv;  // [2][level+1][N]
    const u64* add;   // modes 1, 3: c0 limbs (stride N); mode 2: ct with add_cap
    u64* out;         // ct with out_cap
    int out_cap;
    int add_cap;
    int mode;         // 0 none, 1 rotation addend sigma_g(c0), 2 ct addend, 3 rotation + ct addend
    u32 galois;
    const u64* add2;  // mode 3: ct with add_cap added to both components
};

struct TensorJob {
    const u64* a;
    const u64* b;
    u64* out;  // [3][level+1][N]
    int a_cap, b_cap;
};

// job lists travel as kernel parameters (no descriptor copies, capturable in graphs)
#define FR_MAX_JOBS 64
// jobs grouped by key: group g uses gkey[g] for jobs gstart[g] .. gstart[g+1]-1
struct IPJobs {
    IPJob j[FR_MAX_JOBS];
    const u64* gkey[FR_MAX_JOBS];
    int gstart[FR_MAX_JOBS + 1];
    int ngroups;
};
struct MDJobs { MDJob j[FR_MAX_JOBS]; };
// Inner products summed straight into the accumulators of their sums of rotations: group g
// (jobs gstart[g] .. gstart[g+1]-1) adds into j[gstart[g]].out. Each job's ext, key, galois and
// addb (its rotated ciphertext's c0) are used as in IPJobs.
struct IPSumJobs {
    IPJob j[FR_MAX_JOBS];
    int gstart[FR_MAX_JOBS + 1];
    int ngroups;
};
struct TensorJobs { TensorJob j[FR_MAX_JOBS]; };

// Forward NTT that stores its values in Montgomery form (x 2^64 mod q), in place.
void launch_ntt_tomont(const RingDev& R, const PolyBatch& b, cudaStream_t s);
// Forward NTT of the P -> Q conversions of a ModDown fused with its combine: poly p of b is
// (job p / (2(level+1)), component, limb); the transformed values never reach memory, the
// jobs' outputs do (as launch_moddown_combine would write them).
void launch_ntt_moddown(const RingDev& R, const PolyBatch& b, const MDJobs& jobs, int npos, int level,
                        const u64* pinv, const u64* pinv_s, cudaStream_t s);
// Forward NTT of a rescale's lifted last limb fused with its combine: poly p of b is
// (ct component p / l, limb p % l); writes out = (x - NTT(lifted)) q_l^-1, then mode 1 adds
// the matching component of the ct at add + (p / l / 2) add_bs (cap add_cap), mode 2 doubles
// and subtracts cres[i] from component 0.
// Chebyshev leaves Rescale(T1 cb_j + ca_j) in two launches and one transform, without the
// leaves in memory: launch_leaf_lift forms the lifted last limbs [B nl][2][l][N] from u, the
// coefficient form of T1's last limb ([B][2][N]); launch_ntt_leaf_rescale transforms them
// (b: poly ((b nl + j) 2 + t) l + i) and writes leaf (b, j) at out + (b nl + j) 2 out_cap N.
// T1 of query b at x + b x_bs (cap x_cap); constants [nl][L1] each.
void launch_leaf_lift(const u64* u, const u64* cb, const u64* cb_s, const u64* ca, int nl, int L1, u64* lifted,
                      const RescaleTab* tab, u64 ql, int l, int N, int B, cudaStream_t s);
void launch_ntt_leaf_rescale(const RingDev& R, const PolyBatch& b, const u64* x, long long x_bs, int x_cap,
                             const u64* cb, const u64* cb_s, const u64* ca, int nl, int L1, u64* out, int out_cap,
                             const RescaleTab* tab, int l, cudaStream_t s);
void launch_ntt_rescale(const RingDev& R, const PolyBatch& b, const u64* x, int x_cap, u64* out, int out_cap,
                        const RescaleTab* tab, int l, int mode, const u64* add, int add_cap, long long add_bs,
                        const u64* cres, cudaStream_t s);
// Baby steps kept in Q_l u P: baby 0 = P q (zero on the P positions) of each of B queries,
// babies [B][n1][2][npos][N]; babies 1..n1-1 are inner products with IPJob::addb set.
void launch_baby0_pq(u64* babies, long long baby_q, const u64* q, long long q_bs, int q_cap, int B, int npos,
                     int level, const DevPrime* primes, const u64* pmod, const u64* pmod_s, int N, cudaStream_t s);
// Relinearisation fused with the rescale after it (J products at level l): launch_rs_last forms
// z = acc_l P^-1 + d_l [J][2][N]; after its inverse NTT, launch_rs_lift forms y = conv P^-1 +
// centered lift [J][2][l][N]; the forward NTT of y with launch_ntt_relin_rescale writes
// out_j = (acc P^-1 + d - NTT(y)) q_l^-1 (+ the EpiRescale modes) at level l - 1.
void launch_rs_last(const u64* acc, const u64* d, u64* z, const u64* pinv, const u64* pinv_s, int npos, int l,
                    const DevPrime* primes, int N, int J, cudaStream_t s);
void launch_rs_lift(const u64* zc, const u64* conv, u64* y, const u64* pinv, const u64* pinv_s, const RescaleTab* tab,
                    const DevPrime* primes, int l, int N, int J, cudaStream_t s);
void launch_ntt_relin_rescale(const RingDev& R, const PolyBatch& b, const u64* acc, const u64* d, int npos, int l,
                              const u64* pinv, const u64* pinv_s, const RescaleTab* tab, u64* out, int out_cap,
                              long long out_bs, int mode, const u64* add, int add_cap, long long add_bs,
                              const u64* cres, cudaStream_t s);
// ModUp of J inputs: coefficient form of input j at in + j in_job, evaluation form (for the
// digits' own positions) at in_eval + j eval_job
void launch_modup(const u64* in, long long in_job, const u64* in_eval, long long eval_job, u64* ext,
                  const ModUpTab* tabs, int beta, int npos, int N, int J, cudaStream_t s);
void launch_ip(const IPJobs& jobs, int beta, int npos, int level, int kp, int T, const DevPrime* primes,
               const PrimeMap& pos_prime, int logN, cudaStream_t s, const u64* pmod = nullptr,
               const u64* pmod_s = nullptr);
void launch_p2q(const u64* acc, long long acc_job, int npos, int level, u64* conv, const P2QTab* tab, int N, int J,
                cudaStream_t s);
void launch_moddown_combine(const MDJobs& jobs, int J, int npos, int level, const u64* pinv, const u64* pinv_s,
                            const DevPrime* primes, int logN, cudaStream_t s);
void launch_rescale_lift(const u64* last, u64* lifted, const RescaleTab* tab, int l, int N, int BT, cudaStream_t s);
void launch_rescale_combine(const u64* x, int x_cap, const u64* lifted, u64* out, int out_cap, const RescaleTab* tab,
                            int l, int N, int BT, cudaStream_t s);
void launch_tensor(const TensorJobs& jobs, int J, int level, const DevPrime* primes, int N, cudaStream_t s);
// B <= 4 queries: babies of query b at babies + b * baby_q, outputs at out + b * out_q
// Sums of rotations with one ModDown (double hoisting), without the per-job inner products in
// memory: for each group g and position,
// out_g += sum_{jobs of g} (IP_j + P sigma_j(addb_j) on the Q positions of component 0), the
// inner products as launch_ip computes them. out_g: [2][npos][N], read and written.
void launch_ip_sum(const IPSumJobs& jobs, int beta, int npos, int level, int kp, int T, const DevPrime* primes,
                   const PrimeMap& pos_prime, int logN, const u64* pmod, const u64* pmod_s, cudaStream_t s);
// Encrypted-database MAC: (d0, d1, d2)_j = sum_i B_i (x) E_{j n1 + i} for every giant step j.
// babies [n1][2][cap_b][N]; diags [ell][2][nl][N] (evaluation form, Montgomery); out [n2][3][cap_o][N].
void launch_mac_ct(const u64* babies, int cap_b, const u64* diags, u64* out, int cap_o, int nl, int n1, int n2, int ell,
                   const DevPrime* primes, int N, cudaStream_t s);
// The diagonal MAC of B = 1..4 queries against one database with the diagonals streamed
// through a shared-memory ring of asynchronous copies, every diagonal word read once for all B
// queries (the sums of launch_mac: babies of query b at babies + b baby_q, [n1][2][cap_b][N];
// outputs at out + b out_q, [n2][2][cap_o][N]); usable when mac_pipe_fits.
bool mac_pipe_fits(int n1, int ell, int N);
// The same sums as a persistent pipeline (k_mac_ring): one CTA per GPU slot runs point tiles in
// turn, the next tile's diagonals and babies in flight while this one is multiplied; B = 1..4
// queries, each diagonal word read once for all of them. Usable when mac_ring_fits.
bool mac_ring_fits(int n1, int ell, int N, int B);
void launch_mac_ring(const u64* babies, long long baby_q, int cap_b, const u64* diags, u64* out, long long out_q,
                     int cap_o, int nl, int n1, int ell, int B, const DevPrime* primes, int N, cudaStream_t s);
void launch_mac_pipe(const u64* babies, long long baby_q, int cap_b, const u64* diags, u64* out, long long out_q,
                     int cap_o, int nl, int n1, int ell, int B, const DevPrime* primes, int N, cudaStream_t s);
void launch_mac(const u64* babies, long long baby_q, int cap_b, const u64* diags, u64* out, long long out_q,
                int cap_o, int nl, int n1, int n2, int ell, int B, const DevPrime* primes, int N, cudaStream_t s);
// Table schedule (Algorithm 1): out_g = sum_{m < ell} table[m] (.) D_{g,m} for g < G (evaluation form,
// not rescaled); table [ell][2][cap_t][N], group g's diagonals at diags + g * dgrp.
void launch_mac_table(const u64* table, int cap_t, const u64* diags, long long dgrp, int G, u64* out, int cap_o,
                      long long og, int nl, int ell, const DevPrime* primes, int N, cudaStream_t s);
void launch_add(const u64* a, int a_cap, long long a_bs, const u64* b, int b_cap, long long b_bs, u64* out, int o_cap,
                long long o_bs, int level, int B, const DevPrime* primes, int N, cudaStream_t s);
void launch_sum(const u64* a, int cap, long long js, int J, u64* out, int o_cap, int level, const DevPrime* primes,
                int N, cudaStream_t s);
void launch_to_mont(u64* x, long long n_per_poly, const PrimeMap& pm, const DevPrime* primes, long long total,
                    cudaStream_t s);
void launch_encode_diags(const float* T, long long K, int ell, int logn, long long grp, int d0, int nd, int n1,
                         void* zbuf, u64* out_coeff, int nl, const DevPrime* primes, int scale_bits,
                         const unsigned* rot, const double* zr, const double* zi, cudaStream_t s);
// Storage tier B: the same encoding up to the rounded integer coefficients, out_int [nd][N].
void launch_encode_diags_int(const float* T, long long K, int ell, int logn, long long grp, int d0, int nd, int n1,
                             void* zbuf, long long* out_int, int scale_bits, const unsigned* rot, const double* zr,
                             const double* zi, cudaStream_t s);
// Residues of stored integer coefficients: m [nd][N] -> out [nd][nl][N] (coefficient form).
void launch_coef_residues(const long long* m, int nd, u64* out, int nl, const DevPrime* primes, int N,
                          cudaStream_t s);
