// Host-side ring arithmetic, sampling, encoding, keys and Chebyshev algebra.
// Compiled without floating-point contraction: the encoding FFT and the
// Chebyshev coefficient algebra must produce the same doubles on every host.
#include "fr_host.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>
#include <thread>

namespace frh {

u64 powm(u64 a, u64 e, u64 q) {
    u64 r = 1 % q, b = a % q;
    for (; e; e >>= 1) {
        if (e & 1) r = mulm(r, b, q);
        b = mulm(b, b, q);
    }
    return r;
}

// Deterministic Miller-Rabin; the first twelve primes as witnesses cover all 64-bit n.
bool is_prime(u64 n) {
    const u64 W[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 w : W) {
        if (n % w == 0) return n == w;
    }
    u64 d = n - 1;
    int r = 0;
    while (!(d & 1)) { d >>= 1; ++r; }
    for (u64 w : W) {
        u64 x = powm(w, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int i = 1; i < r && witness; ++i) {
            x = mulm(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

bool gen_primes(int logN, const std::vector<int>& bits, std::vector<u64>& out) {
    const u64 step = (u64)2 << logN;
    out.clear();
    for (int b : bits) {
        if (b < 20 || b > 61) return false;
        const u64 hi = ((u64)1 << b) - 1, lo = (u64)1 << (b - 1);
        u64 cand = hi - ((hi - 1) % step);  // largest value <= hi that is 1 mod step
        bool ok = false;
        for (; cand >= lo; cand -= step) {
            if (std::find(out.begin(), out.end(), cand) != out.end()) continue;
            if (is_prime(cand)) { ok = true; break; }
        }
        if (!ok) return false;
        out.push_back(cand);
    }
    return true;
}

static u64 least_generator(u64 q) {
    std::vector<u64> fac;
    u64 m = q - 1;
    for (u64 f = 2; f * f <= m; f = (f == 2 ? 3 : f + 2)) {
        if (m % f) continue;
        fac.push_back(f);
        while (m % f == 0) m /= f;
    }
    if (m > 1) fac.push_back(m);
    for (u64 g = 2;; ++g) {
        bool gen = true;
        for (u64 f : fac)
            if (powm(g, (q - 1) / f, q) == 1) { gen = false; break; }
        if (gen) return g;
    }
}

static uint32_t bitrev(uint32_t v, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i, v >>= 1) r = (r << 1) | (v & 1);
    return r;
}

int Ring::digits_at(int level) const {
    int b = 0;
    while (b < ndig && dstart[b] <= level) ++b;
    return b;
}
void Ring::digit_range(int level, int d, int* lo, int* hi) const {
    *lo = dstart[d];
    *hi = std::min(dstart[d + 1], level + 1);
}

bool ring_init(Ring& R, int logN, const std::vector<int>& qbits, const std::vector<int>& pbits, int dnum,
               int scale_bits, std::string& err) {
    if (logN < 10 || logN > 16) { err = "log_n must be in [10, 16]"; return false; }
    if (qbits.empty() || pbits.empty() || qbits.size() + pbits.size() > 64) { err = "bad prime counts"; return false; }
    if (dnum < 1) { err = "dnum must be >= 1"; return false; }
    R.logN = logN;
    R.N = 1 << logN;
    R.nq = (int)qbits.size();
    R.np = (int)pbits.size();
    R.scale_bits = scale_bits;
    std::vector<int> bits(qbits);
    bits.insert(bits.end(), pbits.begin(), pbits.end());
    if (!gen_primes(logN, bits, R.primes)) { err = "prime generation failed"; return false; }
    // dnum digits (capped at nq): nq / dnum limbs each, the remainder spread one
    // limb at a time over the last digits
    R.ndig = std::min(dnum, R.nq);
    R.dstart.assign(R.ndig + 1, 0);
    const int base = R.nq / R.ndig, extra = R.nq % R.ndig;
    for (int d = 0; d < R.ndig; ++d)
        R.dstart[d + 1] = R.dstart[d] + base + (d >= R.ndig - extra ? 1 : 0);
    const int N = R.N;
    const u64 M = 2 * (u64)N;
    R.tabs.resize(R.total());
    for (int i = 0; i < R.total(); ++i) {
        PrimeTables& T = R.tabs[i];
        T.q = R.primes[i];
        u64 g = least_generator(T.q);
        T.psi = powm(g, (T.q - 1) / M, T.q);
        u64 ipsi = invm(T.psi, T.q);
        T.ninv = invm((u64)N, T.q);
        T.tw.resize(N); T.tws.resize(N); T.itw.resize(N); T.itws.resize(N);
        // powers in natural order, then scattered to bit-reversed positions
        std::vector<u64> pw(N), ipw(N);
        pw[0] = ipw[0] = 1;
        for (int k = 1; k < N; ++k) {
            pw[k] = mulm(pw[k - 1], T.psi, T.q);
            ipw[k] = mulm(ipw[k - 1], ipsi, T.q);
        }
        for (int k = 0; k < N; ++k) {
            uint32_t e = bitrev((uint32_t)k, logN);
            T.tw[k] = pw[e];
            T.itw[k] = ipw[e];
            T.tws[k] = shoup_quot(T.tw[k], T.q);
            T.itws[k] = shoup_quot(T.itw[k], T.q);
        }
    }
    const int n = N / 2;
    R.rot_group.resize(n);
    u64 g5 = 1;
    for (int j = 0; j < n; ++j) {
        R.rot_group[j] = (uint32_t)g5;
        g5 = g5 * 5 % M;
    }
    R.zr.resize(M);
    R.zi.resize(M);
    for (u64 k = 0; k < M; ++k) {
        double a = 2.0 * M_PI * (double)k / (double)M;
        R.zr[k] = std::cos(a);
        R.zi[k] = std::sin(a);
    }
    return true;
}

void ntt_fwd(const Ring& R, int pi, u64* a) {
    const PrimeTables& T = R.tabs[pi];
    const u64 q = T.q;
    const int N = R.N;
    for (int m = 1, t = N >> 1; m < N; m <<= 1, t >>= 1) {
        for (int i = 0; i < m; ++i) {
            const u64 w = T.tw[m + i], ws = T.tws[m + i];
            u64* x = a + 2 * i * t;
            for (int j = 0; j < t; ++j) {
                u64 u = x[j], v = mul_shoup(x[j + t], w, ws, q);
                x[j] = addm(u, v, q);
                x[j + t] = subm(u, v, q);
            }
        }
    }
}

void ntt_inv(const Ring& R, int pi, u64* a) {
    const PrimeTables& T = R.tabs[pi];
    const u64 q = T.q;
    const int N = R.N;
    for (int m = N >> 1, t = 1; m >= 1; m >>= 1, t <<= 1) {
        for (int i = 0; i < m; ++i) {
            const u64 w = T.itw[m + i], ws = T.itws[m + i];
            u64* x = a + 2 * i * t;
            for (int j = 0; j < t; ++j) {
                u64 u = x[j], v = x[j + t];
                x[j] = addm(u, v, q);
                x[j + t] = mul_shoup(subm(u, v, q), w, ws, q);
            }
        }
    }
    const u64 ns = shoup_quot(T.ninv, q);
    for (int j = 0; j < N; ++j) a[j] = mul_shoup(a[j], T.ninv, ns, q);
}

void automorph_eval(const Ring& R, u64 g, const u64* in, u64* out) {
    const u64 M = 2 * (u64)R.N;
    for (int k = 0; k < R.N; ++k) {
        u64 e = 2 * (u64)bitrev((uint32_t)k, R.logN) + 1;
        u64 e2 = e * g % M;
        out[k] = in[bitrev((uint32_t)((e2 - 1) >> 1), R.logN)];
    }
}

u64 galois_of_rotation(const Ring& R, long k) {
    const long n = R.N / 2;
    long r = k % n;
    if (r < 0) r += n;
    return powm(5, (u64)r, 2 * (u64)R.N);
}

// ---------------------------------------------------------------------------
// ChaCha20 (RFC 8439 Section 2.3) and the samplers.
// Stream of an object: key = (seed lo, seed hi, 0x2d726601, 0...), nonce =
// (object lo, object hi, limb), block counter from 0.
// ---------------------------------------------------------------------------
static inline uint32_t rotl(uint32_t v, int c) { return (v << c) | (v >> (32 - c)); }
static inline void qround(uint32_t* x, int a, int b, int c, int d) {
    x[a] += x[b]; x[d] = rotl(x[d] ^ x[a], 16);
    x[c] += x[d]; x[b] = rotl(x[b] ^ x[c], 12);
    x[a] += x[b]; x[d] = rotl(x[d] ^ x[a], 8);
    x[c] += x[d]; x[b] = rotl(x[b] ^ x[c], 7);
}

void chacha20_block(const uint32_t key[8], uint32_t counter, const uint32_t nonce[3], uint8_t out[64]) {
    uint32_t in[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u};
    for (int i = 0; i < 8; ++i) in[4 + i] = key[i];
    in[12] = counter;
    for (int i = 0; i < 3; ++i) in[13 + i] = nonce[i];
    uint32_t x[16];
    std::memcpy(x, in, sizeof(x));
    for (int round = 0; round < 10; ++round) {
        qround(x, 0, 4, 8, 12); qround(x, 1, 5, 9, 13); qround(x, 2, 6, 10, 14); qround(x, 3, 7, 11, 15);
        qround(x, 0, 5, 10, 15); qround(x, 1, 6, 11, 12); qround(x, 2, 7, 8, 13); qround(x, 3, 4, 9, 14);
    }
    for (int i = 0; i < 16; ++i) {
        uint32_t v = x[i] + in[i];
        for (int b = 0; b < 4; ++b) out[4 * i + b] = (uint8_t)(v >> (8 * b));
    }
}

namespace {
class Stream {
   public:
    Stream(u64 seed, u64 obj, uint32_t limb) {
        key_[0] = (uint32_t)seed;
        key_[1] = (uint32_t)(seed >> 32);
        key_[2] = 0x2d726601u;
        for (int i = 3; i < 8; ++i) key_[i] = 0;
        nonce_[0] = (uint32_t)obj;
        nonce_[1] = (uint32_t)(obj >> 32);
        nonce_[2] = limb;
    }
    uint8_t byte() {
        if (pos_ == 64) {
            chacha20_block(key_, ctr_++, nonce_, buf_);
            pos_ = 0;
        }
        return buf_[pos_++];
    }
    u64 le(int nbytes) {
        u64 v = 0;
        for (int i = 0; i < nbytes; ++i) v |= (u64)byte() << (8 * i);
        return v;
    }

   private:
    uint32_t key_[8], nonce_[3], ctr_ = 0;
    uint8_t buf_[64];
    int pos_ = 64;
};
}  // namespace

void sample_ternary(u64 seed, u64 obj, int n, int8_t* out) {
    Stream st(seed, obj, 0);
    for (int i = 0; i < n; ++i) {
        uint8_t b = st.byte();
        while (b == 255) b = st.byte();
        out[i] = (int8_t)(b % 3) - 1;
    }
}

void sample_cbd(u64 seed, u64 obj, int n, int32_t* out) {
    Stream st(seed, obj, 0);
    const u64 m21 = (1ull << 21) - 1;
    for (int i = 0; i < n; ++i) {
        u64 v = st.le(6);
        out[i] = __builtin_popcountll(v & m21) - __builtin_popcountll((v >> 21) & m21);
    }
}

void sample_uniform(u64 seed, u64 obj, uint32_t limb, u64 q, int n, u64* out) {
    Stream st(seed, obj, limb);
    int bl = 64 - __builtin_clzll(q);
    const u64 mask = bl >= 64 ? ~0ull : ((1ull << bl) - 1);
    for (int i = 0; i < n; ++i) {
        u64 v;
        do { v = st.le(8) & mask; } while (v >= q);
        out[i] = v;
    }
}

// ---------------------------------------------------------------------------
// Slot encoding: inverse special FFT in the 5^j slot order, times 1/n and the
// scale, rounded half away from zero. Stage order and complex products are
// fixed (the device encoder performs the same operations).
// ---------------------------------------------------------------------------
static void bitrev_permute(std::vector<double>& re, std::vector<double>& im) {
    const int n = (int)re.size();
    int lg = 0;
    while ((1 << lg) < n) ++lg;
    for (int i = 0; i < n; ++i) {
        int j = (int)bitrev((uint32_t)i, lg);
        if (i < j) { std::swap(re[i], re[j]); std::swap(im[i], im[j]); }
    }
}

void encode_coeffs(const Ring& R, const double* z, int scale_bits, int64_t* m) {
    const int n = R.N / 2;
    const u64 M = 2 * (u64)R.N;
    std::vector<double> re(z, z + n), im(n, 0.0);
    for (int len = n; len >= 2; len >>= 1) {
        const int h = len >> 1;
        const u64 lq = (u64)len << 2, gap = M / lq;
        for (int base = 0; base < n; base += len) {
            for (int j = 0; j < h; ++j) {
                const u64 idx = (lq - R.rot_group[j] % lq) * gap;
                const double wr = R.zr[idx], wi = R.zi[idx];
                double* a_r = &re[base + j]; double* a_i = &im[base + j];
                double* b_r = &re[base + j + h]; double* b_i = &im[base + j + h];
                const double sr = *a_r + *b_r, si = *a_i + *b_i;
                const double dr = *a_r - *b_r, di = *a_i - *b_i;
                *a_r = sr;
                *a_i = si;
                *b_r = dr * wr - di * wi;
                *b_i = dr * wi + di * wr;
            }
        }
    }
    bitrev_permute(re, im);
    const double inv_n = 1.0 / (double)n, delta = std::ldexp(1.0, scale_bits);
    for (int k = 0; k < n; ++k) {
        m[k] = std::llround((re[k] * inv_n) * delta);
        m[k + n] = std::llround((im[k] * inv_n) * delta);
    }
}

void decode_coeffs(const Ring& R, const int64_t* x, double scale, double* z) {
    std::vector<double> v(x, x + R.N);
    decode_values(R, v.data(), scale, z);
}

void decode_values(const Ring& R, const double* x, double scale, double* z) {
    const int n = R.N / 2;
    const u64 M = 2 * (u64)R.N;
    std::vector<double> re(n), im(n);
    for (int k = 0; k < n; ++k) { re[k] = x[k]; im[k] = x[k + n]; }
    bitrev_permute(re, im);
    for (int len = 2; len <= n; len <<= 1) {
        const int h = len >> 1;
        const u64 lq = (u64)len << 2, gap = M / lq;
        for (int base = 0; base < n; base += len) {
            for (int j = 0; j < h; ++j) {
                const u64 idx = (R.rot_group[j] % lq) * gap;
                const double wr = R.zr[idx], wi = R.zi[idx];
                const double br = re[base + j + h], bi = im[base + j + h];
                const double vr = br * wr - bi * wi, vi = br * wi + bi * wr;
                const double ar = re[base + j], ai = im[base + j];
                re[base + j] = ar + vr;
                im[base + j] = ai + vi;
                re[base + j + h] = ar - vr;
                im[base + j + h] = ai - vi;
            }
        }
    }
    for (int j = 0; j < n; ++j) z[j] = re[j] / scale;
}

// ---------------------------------------------------------------------------
// Keys
// ---------------------------------------------------------------------------
namespace {
const u64 kObjS = 0x01, kObjPkA = 0x02, kObjPkE = 0x03;
const u64 kObjEncV = 0x11, kObjEncE0 = 0x12, kObjEncE1 = 0x13;
u64 evk_obj(bool relin, u64 g, int d, int part) {
    return ((u64)(relin ? 2 : 1) << 40) | ((relin ? 0 : g) << 8) | ((u64)d << 1) | (u64)part;
}

template <class F>
void parallel_for(int n, int nthreads, F f) {
    if (nthreads <= 1 || n <= 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> th;
    int nt = std::min(nthreads, n);
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            for (int i = t; i < n; i += nt) f(i);
        });
    for (auto& x : th) x.join();
}

// hybrid key-switching key for s' = sigma_g(s) (relin == false) or s^2 (relin == true)
void make_ksk(const Ring& R, const KeySet& K, bool relin, u64 g, std::vector<u64>& out, int nthreads) {
    const int N = R.N, T = R.total();
    out.assign((size_t)R.ndig * 2 * T * N, 0);
    std::vector<u64> Pmod(T);
    for (int i = 0; i < T; ++i) {
        u64 v = 1;
        for (int j = 0; j < R.np; ++j) v = mulm(v, R.primes[R.nq + j] % R.primes[i], R.primes[i]);
        Pmod[i] = v;
    }
    for (int d = 0; d < R.ndig; ++d) {
        std::vector<int32_t> e(N);
        sample_cbd(K.seed, evk_obj(relin, g, d, 1), N, e.data());
        parallel_for(T, nthreads, [&](int i) {
            const u64 q = R.primes[i];
            u64* b = &out[(((size_t)d * 2 + 0) * T + i) * N];
            u64* a = &out[(((size_t)d * 2 + 1) * T + i) * N];
            const u64* se = &K.s_eval[(size_t)i * N];
            sample_uniform(K.seed, evk_obj(relin, g, d, 0), (uint32_t)i, q, N, a);
            for (int j = 0; j < N; ++j) b[j] = resid(e[j], q);
            ntt_fwd(R, i, b);
            std::vector<u64> sp(N);
            if (relin) {
                for (int j = 0; j < N; ++j) sp[j] = mulm(se[j], se[j], q);
            } else {
                automorph_eval(R, g, se, sp.data());
            }
            const bool mine = i >= R.dstart[d] && i < R.dstart[d + 1];
            for (int j = 0; j < N; ++j) {
                u64 v = subm(b[j], mulm(a[j], se[j], q), q);
                if (mine) v = addm(v, mulm(Pmod[i], sp[j], q), q);
                b[j] = v;
            }
        });
    }
}
}  // namespace

void keygen(const Ring& R, u64 seed, const std::vector<u64>& galois, KeySet& K, int nthreads) {
    const int N = R.N, T = R.total();
    K.seed = seed;
    K.s.resize(N);
    sample_ternary(seed, kObjS, N, K.s.data());
    K.s_eval.resize((size_t)T * N);
    parallel_for(T, nthreads, [&](int i) {
        u64* r = &K.s_eval[(size_t)i * N];
        for (int j = 0; j < N; ++j) r[j] = resid(K.s[j], R.primes[i]);
        ntt_fwd(R, i, r);
    });
    K.pk0.resize((size_t)R.nq * N);
    K.pk1.resize((size_t)R.nq * N);
    std::vector<int32_t> e(N);
    sample_cbd(seed, kObjPkE, N, e.data());
    parallel_for(R.nq, nthreads, [&](int i) {
        const u64 q = R.primes[i];
        u64* a = &K.pk1[(size_t)i * N];
        u64* b = &K.pk0[(size_t)i * N];
        sample_uniform(seed, kObjPkA, (uint32_t)i, q, N, a);
        for (int j = 0; j < N; ++j) b[j] = resid(e[j], q);
        ntt_fwd(R, i, b);
        const u64* se = &K.s_eval[(size_t)i * N];
        for (int j = 0; j < N; ++j) b[j] = subm(b[j], mulm(a[j], se[j], q), q);
    });
    make_ksk(R, K, true, 0, K.relin, nthreads);
    K.rot.clear();
    for (u64 g : galois) {
        bool dup = false;
        for (auto& kv : K.rot) dup |= kv.first == g;
        if (dup || g == 1) continue;
        K.rot.emplace_back(g, std::vector<u64>());
        make_ksk(R, K, false, g, K.rot.back().second, nthreads);
    }
}

void encrypt(const Ring& R, const KeySet& K, const double* z, u64 seed, u64* out) {
    encrypt_level(R, K, z, seed, R.nq - 1, (int)std::thread::hardware_concurrency(), out);
}

void encrypt_level(const Ring& R, const KeySet& K, const double* z, u64 seed, int level, int nthreads, u64* out) {
    const int N = R.N, nq = level + 1;
    std::vector<int64_t> m(N);
    encode_coeffs(R, z, R.scale_bits, m.data());
    std::vector<int8_t> v(N);
    std::vector<int32_t> e0(N), e1(N);
    sample_ternary(seed, kObjEncV, N, v.data());
    sample_cbd(seed, kObjEncE0, N, e0.data());
    sample_cbd(seed, kObjEncE1, N, e1.data());
    parallel_for(nq, nthreads, [&](int i) {
        const u64 q = R.primes[i];
        std::vector<u64> V(N);
        for (int j = 0; j < N; ++j) V[j] = resid(v[j], q);
        ntt_fwd(R, i, V.data());
        u64* c0 = out + (size_t)i * N;
        u64* c1 = out + ((size_t)nq + i) * N;
        for (int j = 0; j < N; ++j) {
            c0[j] = mulm(V[j], K.pk0[(size_t)i * N + j], q);
            c1[j] = mulm(V[j], K.pk1[(size_t)i * N + j], q);
        }
        ntt_inv(R, i, c0);
        ntt_inv(R, i, c1);
        for (int j = 0; j < N; ++j) {
            c0[j] = addm(addm(c0[j], resid(e0[j], q), q), resid(m[j], q), q);
            c1[j] = addm(c1[j], resid(e1[j], q), q);
        }
    });
}

void encrypt_diagonals(const Ring& R, const KeySet& K, const float* T, long long rows, int ell, int n1, bool prerotate,
                       int level, u64 seed, int nthreads, u64* out) {
    const int n = R.N / 2;
    const long long G = (rows + n - 1) / n, B = n / ell;
    const size_t cw = (size_t)2 * (level + 1) * R.N;
    parallel_for((int)(G * ell), nthreads, [&](int e) {
        const long long g = e / ell;
        const int d = e % ell;
        const long long shift = prerotate ? (long long)(d / n1) * n1 : 0;
        std::vector<double> z(n);
        for (int x = 0; x < n; ++x) {
            const long long y = ((x - shift) % n + n) % n;
            const long long row = (g * B + y / ell) * ell + y % ell;
            z[x] = row < rows ? (double)T[(size_t)row * ell + (size_t)((y % ell + d) % ell)] : 0.0;
        }
        encrypt_level(R, K, z.data(), seed + (u64)e, level, 1, out + (size_t)e * cw);
    });
}

void decrypt_coeffs(const Ring& R, const KeySet& K, const u64* ct, int level, int64_t* x) {
    const int N = R.N;
    const u64 q = R.primes[0];
    std::vector<u64> a(ct + (size_t)(level + 1) * N, ct + (size_t)(level + 2) * N);
    ntt_fwd(R, 0, a.data());
    for (int j = 0; j < N; ++j) a[j] = mulm(a[j], K.s_eval[j], q);
    ntt_inv(R, 0, a.data());
    for (int j = 0; j < N; ++j) {
        u64 v = addm(a[j], ct[j], q);
        x[j] = v > (q - 1) / 2 ? -(int64_t)(q - v) : (int64_t)v;
    }
}

void decrypt_values(const Ring& R, const KeySet& K, const u64* ct, int level, double* x) {
    const int N = R.N;
    const int nl = level >= 1 ? 2 : 1;
    std::vector<std::vector<u64>> m(nl);
    for (int i = 0; i < nl; ++i) {
        const u64 q = R.primes[i];
        m[i].assign(ct + (size_t)(level + 1 + i) * N, ct + (size_t)(level + 2 + i) * N);
        ntt_fwd(R, i, m[i].data());
        for (int j = 0; j < N; ++j) m[i][j] = mulm(m[i][j], K.s_eval[(size_t)i * N + j], q);
        ntt_inv(R, i, m[i].data());
        for (int j = 0; j < N; ++j) m[i][j] = addm(m[i][j], ct[(size_t)i * N + j], q);
    }
    const u64 q0 = R.primes[0];
    if (nl == 1) {
        for (int j = 0; j < N; ++j) x[j] = m[0][j] > (q0 - 1) / 2 ? -(double)(q0 - m[0][j]) : (double)m[0][j];
        return;
    }
    const u64 q1 = R.primes[1];
    const u64 q0inv = invm(q0 % q1, q1);
    const u128 Q = (u128)q0 * q1;
    for (int j = 0; j < N; ++j) {
        // x = m0 + q0 * ((m1 - m0) q0^-1 mod q1), centered in (-Q/2, Q/2]
        const u64 h = mulm(subm(m[1][j], m[0][j] % q1, q1), q0inv, q1);
        const u128 y = (u128)m[0][j] + (u128)q0 * h;
        x[j] = y > (Q - 1) / 2 ? -(double)(Q - y) : (double)y;
    }
}

// ---------------------------------------------------------------------------
// Chebyshev algebra
// ---------------------------------------------------------------------------
void cheb_coeffs(int n, double tau, std::vector<double>& c, double low) {
    c.assign(n + 1, 0.0);
    for (int k = 0; k <= n; ++k) {
        double acc = 0.0;
        for (int j = 0; j <= n; ++j) {
            const double th = M_PI * ((double)j + 0.5) / (double)(n + 1);
            const double fx = std::cos(th) >= tau ? 1.0 : low;
            acc = acc + fx * std::cos((double)k * th);
        }
        c[k] = acc * ((k == 0 ? 1.0 : 2.0) / (double)(n + 1));
    }
}

void ps_split(int n, int* d1, int* d2) {
    int best = 1 << 30;
    *d1 = *d2 = 0;
    for (int a = 1; a <= n + 1; ++a) {
        int b = 1;
        while ((double)a * std::ldexp(1.0, b - 1) < (double)n) ++b;
        if (a + b < best || (a + b == best && a > *d1)) {
            best = a + b;
            *d1 = a;
            *d2 = b;
        }
    }
}

void cheb_split(const std::vector<double>& c, std::vector<double>& q, std::vector<double>& r) {
    const int M = (int)c.size() / 2;
    q.assign(M, 0.0);
    r.assign(M, 0.0);
    q[0] = c[M];
    r[0] = c[0];
    for (int i = 1; i < M; ++i) {
        q[i] = 2.0 * c[M + i];
        r[i] = c[i] - c[2 * M - i];
    }
}

void bconv_consts(const Ring& R, const std::vector<int>& src, int tgt_prime, std::vector<u64>& inv_hat,
                  std::vector<u64>& hat_t) {
    const u64 t = R.primes[tgt_prime];
    inv_hat.resize(src.size());
    hat_t.resize(src.size());
    for (size_t i = 0; i < src.size(); ++i) {
        const u64 bi = R.primes[src[i]];
        u64 h = 1, ht = 1;
        for (size_t j = 0; j < src.size(); ++j) {
            if (j == i) continue;
            h = mulm(h, R.primes[src[j]] % bi, bi);
            ht = mulm(ht, R.primes[src[j]] % t, t);
        }
        inv_hat[i] = invm(h, bi);
        hat_t[i] = ht;
    }
}

// Rotation index sets of the schemes compared in the paper (Section "Complexity
// analysis and memory consumption", GPU complexity table) and of this build.
bool rotation_set(uint32_t ell, uint32_t n1, uint32_t slots, int variant, bool membership, std::vector<long>& out) {
    if (ell == 0 || n1 == 0 || n1 > ell || slots == 0 || (slots & (slots - 1))) return false;
    const long n2 = (ell + n1 - 1) / n1;
    std::set<long> s;
    auto baby = [&] { for (long i = 1; i < (long)n1; ++i) s.insert(i); };
    auto giant = [&](long sign) { for (long j = 1; j < n2; ++j) s.insert(sign * j * (long)n1); };
    auto pow2 = [&] { for (long p = 1; p < (long)slots; p <<= 1) s.insert(p); };
    switch (variant) {
        case RV_ONDEMAND:
        case RV_TABLE:
            baby(); giant(1);
            if (membership) pow2();
            break;
        case RV_CPU_BSGS: baby(); giant(1); break;
        case RV_HYDIA_DG:
            for (long i = 1; i < (long)ell; ++i) s.insert(i);
            pow2();
            break;
        case RV_TBS_ONLINE: giant(1); pow2(); break;
        case RV_TBS_TOTAL: baby(); giant(1); giant(-1); pow2(); break;
        case RV_TBE_TOTAL: baby(); giant(1); pow2(); break;
        default: return false;
    }
    out.assign(s.begin(), s.end());
    return true;
}

int plan_batch(const uint32_t* cls, size_t n, uint32_t max_batch, uint64_t avail, uint64_t ws_base,
               uint64_t ws_per_query, uint32_t* idx) {
    if (n == 0 || max_batch == 0) return 0;
    uint32_t cnt = 0;
    for (size_t i = 0; i < n && cnt < max_batch; ++i)
        if (cls[i] == cls[0]) idx[cnt++] = (uint32_t)i;
    uint32_t B = 1;
    while (B * 2 <= cnt) B *= 2;
    while (B > 0 && ws_base + (uint64_t)B * ws_per_query > avail) B /= 2;
    return (int)B;
}

}  // namespace frh
