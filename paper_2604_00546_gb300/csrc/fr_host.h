// Host-side (client and set-up) part of the library: prime chain, NTT tables,
// ChaCha20 sampling, slot encoding, key generation, encryption, decryption,
// Chebyshev coefficient algebra and rotation-set bookkeeping.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace frh {

typedef uint64_t u64;
typedef unsigned __int128 u128;

inline u64 mulm(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
inline u64 addm(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
inline u64 subm(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }
u64 powm(u64 a, u64 e, u64 q);
inline u64 invm(u64 a, u64 q) { return powm(a % q, q - 2, q); }
inline u64 shoup_quot(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }
inline u64 mul_shoup(u64 x, u64 w, u64 ws, u64 q) {
    u64 hi = (u64)(((u128)x * ws) >> 64);
    u64 r = x * w - hi * q;
    return r >= q ? r - q : r;
}
inline u64 resid(int64_t v, u64 q) {
    if (v >= 0) return (u64)v % q;
    u64 a = (u64)(-(v + 1)) % q;  // v = -(a + 1)
    return q - 1 - a;
}

bool is_prime(u64 n);
// primes = 1 mod 2N, per bit size largest first, in the order of `bits`
bool gen_primes(int logN, const std::vector<int>& bits, std::vector<u64>& out);

// Ring tables of one prime: psi^brev(k), psi^-brev(k) and Shoup quotients.
struct PrimeTables {
    u64 q, psi, ninv;
    std::vector<u64> tw, tws, itw, itws;
};

struct Ring {
    int logN = 0, N = 0;
    int nq = 0, np = 0;                 // Q limbs, P limbs
    int ndig = 0;                       // key-switching digits at the top level
    std::vector<int> dstart;            // digit d = Q limbs [dstart[d], dstart[d+1])
    int scale_bits = 0;
    std::vector<u64> primes;            // Q then P
    std::vector<PrimeTables> tabs;
    std::vector<uint32_t> rot_group;    // 5^j mod 2N, j < N/2
    std::vector<double> zr, zi;         // exp(2 pi i k / 2N)
    int total() const { return nq + np; }
    int digits_at(int level) const;
    void digit_range(int level, int d, int* lo, int* hi) const;
};

bool ring_init(Ring& R, int logN, const std::vector<int>& qbits, const std::vector<int>& pbits, int dnum,
               int scale_bits, std::string& err);
void ntt_fwd(const Ring& R, int pi, u64* a);
void ntt_inv(const Ring& R, int pi, u64* a);
void automorph_eval(const Ring& R, u64 g, const u64* in, u64* out);
u64 galois_of_rotation(const Ring& R, long k);

// ChaCha20 keystream samplers (RFC 8439 block function)
void chacha20_block(const uint32_t key[8], uint32_t counter, const uint32_t nonce[3], uint8_t out[64]);
void sample_ternary(u64 seed, u64 obj, int n, int8_t* out);
void sample_cbd(u64 seed, u64 obj, int n, int32_t* out);
void sample_uniform(u64 seed, u64 obj, uint32_t limb, u64 q, int n, u64* out);

// slot encoding of n = N/2 real values at scale 2^scale_bits into integer coefficients
void encode_coeffs(const Ring& R, const double* z, int scale_bits, int64_t* m);
void decode_coeffs(const Ring& R, const int64_t* x, double scale, double* z);
void decode_values(const Ring& R, const double* x, double scale, double* z);

// Keys. Key-switching keys are [ndig][2][nq+np][N] in evaluation form.
struct KeySet {
    u64 seed = 0;
    std::vector<int8_t> s;
    std::vector<u64> s_eval;   // [nq+np][N]
    std::vector<u64> pk0, pk1; // [nq][N] evaluation form
    std::vector<std::pair<u64, std::vector<u64>>> rot;  // (galois element, key)
    std::vector<u64> relin;
};
void keygen(const Ring& R, u64 seed, const std::vector<u64>& galois, KeySet& K, int nthreads);
void encrypt(const Ring& R, const KeySet& K, const double* z, u64 seed, u64* out /*[2][nq][N] coeff*/);
// limbs 0..level of the top-level encryption with the same seed ([2][level+1][N] coefficient form)
void encrypt_level(const Ring& R, const KeySet& K, const double* z, u64 seed, int level, int nthreads, u64* out);
// Enrollment of an encrypted database: the G ell diagonals of the rows x ell matrix T, each
// pre-rotated by -(d / n1) n1 slots when prerotate is set (plain otherwise) and encrypted at
// `level` with seed + g ell + d, written [G][ell][2][level+1][N] (coefficient form).
void encrypt_diagonals(const Ring& R, const KeySet& K, const float* T, long long rows, int ell, int n1, bool prerotate,
                       int level, u64 seed, int nthreads, u64* out);
void decrypt_coeffs(const Ring& R, const KeySet& K, const u64* ct, int level, int64_t* x);
// plaintext coefficients as reals: centered CRT of limbs 0 and 1 (level >= 1) or limb 0
void decrypt_values(const Ring& R, const KeySet& K, const u64* ct, int level, double* x);

// Chebyshev interpolant of step(x - tau) at n+1 Chebyshev nodes; PS split.
// interpolant at the n + 1 Chebyshev nodes of f = 1 for x >= tau, `low` below (0: step, -1: sign)
void cheb_coeffs(int n, double tau, std::vector<double>& c, double low = 0.0);
void ps_split(int n, int* d1, int* d2);
// Chebyshev division p = q T_M + r (length 2M -> two of length M)
void cheb_split(const std::vector<double>& c, std::vector<double>& q, std::vector<double>& r);

// FastBConv constants: [(B/b_i)^-1]_{b_i} and [B/b_i]_t
void bconv_consts(const Ring& R, const std::vector<int>& src, int tgt_prime, std::vector<u64>& inv_hat,
                  std::vector<u64>& hat_t);

// rotation-set bookkeeping
enum RotVariant { RV_ONDEMAND = 0, RV_CPU_BSGS = 1, RV_HYDIA_DG = 2, RV_TBS_ONLINE = 3, RV_TBS_TOTAL = 4,
                  RV_TBE_TOTAL = 5, RV_TABLE = 6 };
bool rotation_set(uint32_t ell, uint32_t n1, uint32_t slots, int variant, bool membership, std::vector<long>& out);

// Continuous-batching planner. Pending requests are given by class id (one class per
// (database, mode)) in arrival order. The next batch serves the oldest request's class:
// up to max_batch requests of that class in arrival order, the count rounded down to a
// power of two, then halved while ws_base + B ws_per_query exceeds avail. Returns B
// (0 when not even one request fits) and writes the chosen indices to idx.
int plan_batch(const uint32_t* cls, size_t n, uint32_t max_batch, uint64_t avail, uint64_t ws_base,
               uint64_t ws_per_query, uint32_t* idx);

}  // namespace frh
