/*
 * CPU oracle for the encrypted 1:N face-matching hot path of "Lightweight,
 * Practical Encrypted Face Recognition with GPU Support" (arXiv 2604.00546).
 *
 * THIS FILE IS TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / --impl reference legs may load it. The product
 * path (paper_2604_00546_gb300) never imports, links or calls it, and shares
 * no code, tables or constant generators with it.
 *
 * Style: plain and slow on purpose. Every modular product is a 128-bit
 * product reduced with '%'. Ciphertexts are kept in coefficient form; the NTT
 * is used only as the library primitive that multiplies ring elements. Each
 * function names the passage of the paper (section / equation / algorithm)
 * it follows; where the paper is silent, the reading adopted is stated and
 * the same reading is listed in the design notes of the repository.
 *
 * Conventions (the readings shared with the product path, stated once):
 *  - R = Z[X]/(X^N+1), slots n = N/2, M = 2N, slot j <-> zeta^(5^j mod M),
 *    zeta = exp(2*pi*i/M)   (Section "CKKS", encoding paragraph).
 *  - Rot_k is a LEFT rotation: (Rot_k z)[j] = z[(j+k) mod n], realised by the
 *    automorphism X -> X^(5^k mod M) (Section "Diagonal method", Eq. equ:diag
 *    pairs diag_i[r] with v[r+i]).
 *  - Evaluation ("NTT") form of a limb: position k holds A(psi^(2*brev(k)+1)),
 *    psi = g^((q-1)/M), g the smallest generator of Z_q^*.
 *  - Ciphertext (c0, c1) decrypts as c0 + c1*s.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t u64;
typedef uint32_t u32;
typedef unsigned __int128 u128;

#define OR_MAXP 64

/* ------------------------------------------------------------------------ */
/* Modular arithmetic: the plain definitions.                                */
/* ------------------------------------------------------------------------ */
static inline u64 mmul(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static inline u64 madd(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static inline u64 msub(u64 a, u64 b, u64 q) { return (u64)(((u128)a + q - (b % q)) % q); }
static u64 mpow(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mmul(r, a, q);
        a = mmul(a, a, q);
        e >>= 1;
    }
    return r;
}
static u64 minv(u64 a, u64 q) { return mpow(a, q - 2, q); } /* q prime */
/* residue of a signed integer */
static inline u64 mred_s(int64_t v, u64 q) {
    if (v >= 0) return (u64)v % q;
    u64 r = ((u64)(-(v + 1)) % q);       /* -(v+1) >= 0 avoids INT64_MIN overflow */
    return (q - 1 - r) % q;              /* v = -(r'+1) -> q-1-r' */
}

/* ------------------------------------------------------------------------ */
/* Primes (reading R1): primes = 1 mod 2N, taken largest-first per bit size, */
/* Q list first, then P list. Deterministic Miller-Rabin, 12 prime bases.     */
/* ------------------------------------------------------------------------ */
static int is_prime_u64(u64 n) {
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = mpow(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int r = 1; r < s; r++) {
            x = mmul(x, x, n);
            if (x == n - 1) { comp = 0; break; }
        }
        if (comp) return 0;
    }
    return 1;
}

int or_is_prime(u64 n) { return is_prime_u64(n); }

/* bits[i] for i < count; fills out[i]. Returns 0 on success. */
int or_gen_primes(int log_n, const int* bits, int count, u64* out) {
    u64 m = (u64)2 << log_n;
    for (int idx = 0; idx < count; idx++) {
        int b = bits[idx];
        if (b < 20 || b > 61) return -1;
        u64 top = (b == 64) ? ~(u64)0 : (((u64)1 << b) - 1);
        u64 lo = (u64)1 << (b - 1);
        u64 c = (top / m) * m + 1;
        if (c > top) c -= m;
        int found = 0;
        while (c >= lo) {
            int taken = 0;
            for (int t = 0; t < idx; t++)
                if (out[t] == c) taken = 1;
            if (!taken && is_prime_u64(c)) { out[idx] = c; found = 1; break; }
            c -= m;
        }
        if (!found) return -2;
    }
    return 0;
}

/* smallest generator of Z_q^* (q prime), by trial factoring of q-1 */
static u64 smallest_generator(u64 q) {
    u64 f[64];
    int nf = 0;
    u64 r = q - 1;
    for (u64 d = 2; d * d <= r; d += (d == 2 ? 1 : 2)) {
        if (r % d == 0) {
            f[nf++] = d;
            while (r % d == 0) r /= d;
        }
    }
    if (r > 1) f[nf++] = r;
    for (u64 g = 2; g < q; g++) {
        int ok = 1;
        for (int i = 0; i < nf; i++)
            if (mpow(g, (q - 1) / f[i], q) == 1) { ok = 0; break; }
        if (ok) return g;
    }
    return 0;
}

static u32 brev(u32 x, int bits) {
    u32 r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Context                                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int log_n, n, nq, np, dnum, alpha, scale_bits;
    int ndig;                /* key-switching digits at the top level */
    int dstart[OR_MAXP + 1]; /* digit d holds Q limbs [dstart[d], dstart[d+1]) */
    u64 p[OR_MAXP];          /* Q primes (0..nq-1) then P primes (nq..nq+np-1) */
    u64 psi[OR_MAXP];
    u64* psi_rev[OR_MAXP];   /* psi^brev(k) */
    u64* ipsi_rev[OR_MAXP];  /* psi^-brev(k) */
    u64 ninv[OR_MAXP];
    u32* rot_group;          /* 5^j mod M, j < n/2 */
    double* zr;              /* cos(2 pi k / M) */
    double* zi;              /* sin(2 pi k / M) */
    int nthreads;
} or_ctx;

typedef struct {
    u64 seed;
    int8_t* s;      /* ternary secret, coefficient form */
    u64* s_eval;    /* [nq+np][N] evaluation form */
    u64* pk0;       /* [nq][N] evaluation form */
    u64* pk1;
    u64* relin;     /* cached relinearisation key [beta][2][nq+np][N] (eval) */
} or_keys;

int or_n(const or_ctx* c) { return c->n; }
int or_nq(const or_ctx* c) { return c->nq; }
int or_np(const or_ctx* c) { return c->np; }
int or_alpha(const or_ctx* c) { return c->alpha; }
u64 or_prime(const or_ctx* c, int i) { return c->p[i]; }
u64 or_psi(const or_ctx* c, int i) { return c->psi[i]; }

void or_free(or_ctx* c) {
    if (!c) return;
    for (int i = 0; i < c->nq + c->np; i++) { free(c->psi_rev[i]); free(c->ipsi_rev[i]); }
    free(c->rot_group); free(c->zr); free(c->zi);
    free(c);
}

/* Parameters: log_n, Q bit sizes, P bit sizes, dnum (key-switch digits, reading
 * R3: alpha = ceil(nq/dnum) limbs per digit), scale Delta = 2^scale_bits. */
or_ctx* or_setup(int log_n, const int* q_bits, int nq, const int* p_bits, int np, int dnum,
                 int scale_bits) {
    if (log_n < 2 || log_n > 17 || nq < 1 || np < 1 || nq + np > OR_MAXP || dnum < 1) return NULL;
    or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
    c->log_n = log_n;
    c->n = 1 << log_n;
    c->nq = nq;
    c->np = np;
    c->dnum = dnum;
    /* reading R3: dnum digits (at most nq) of floor(nq/dnum) limbs, the
     * remainder given one extra limb each, starting from the LAST digit */
    c->ndig = dnum < nq ? dnum : nq;
    {
        int base = nq / c->ndig, extra = nq % c->ndig, pos = 0;
        for (int d = 0; d < c->ndig; d++) {
            c->dstart[d] = pos;
            pos += base + ((d >= c->ndig - extra) ? 1 : 0);
        }
        c->dstart[c->ndig] = nq;
    }
    c->alpha = nq / c->ndig + (nq % c->ndig ? 1 : 0); /* largest digit size */
    c->scale_bits = scale_bits;
    int bits[OR_MAXP];
    for (int i = 0; i < nq; i++) bits[i] = q_bits[i];
    for (int i = 0; i < np; i++) bits[nq + i] = p_bits[i];
    if (or_gen_primes(log_n, bits, nq + np, c->p) != 0) { free(c); return NULL; }
    int N = c->n;
    u64 M = 2 * (u64)N;
    for (int i = 0; i < nq + np; i++) {
        u64 q = c->p[i];
        u64 g = smallest_generator(q);
        u64 psi = mpow(g, (q - 1) / M, q);
        c->psi[i] = psi;
        u64 ipsi = minv(psi, q);
        c->psi_rev[i] = (u64*)malloc(sizeof(u64) * N);
        c->ipsi_rev[i] = (u64*)malloc(sizeof(u64) * N);
        for (int k = 0; k < N; k++) {
            u32 e = brev((u32)k, log_n);
            c->psi_rev[i][k] = mpow(psi, e, q);
            c->ipsi_rev[i][k] = mpow(ipsi, e, q);
        }
        c->ninv[i] = minv((u64)N % q, q);
    }
    int n = N / 2;
    c->rot_group = (u32*)malloc(sizeof(u32) * (n > 0 ? n : 1));
    u64 g5 = 1;
    for (int j = 0; j < n; j++) { c->rot_group[j] = (u32)g5; g5 = (g5 * 5) % M; }
    c->zr = (double*)malloc(sizeof(double) * M);
    c->zi = (double*)malloc(sizeof(double) * M);
    for (u64 k = 0; k < M; k++) {
        double ang = 2.0 * M_PI * (double)k / (double)M;
        c->zr[k] = cos(ang);
        c->zi[k] = sin(ang);
    }
#ifdef _OPENMP
    c->nthreads = omp_get_max_threads();
#else
    c->nthreads = 1;
#endif
    return c;
}

/* ------------------------------------------------------------------------ */
/* NTT: textbook iterative Cooley-Tukey (forward, bit-reversed output) and    */
/* Gentleman-Sande (inverse) negacyclic transforms. Output position k holds   */
/* A(psi^(2 brev(k)+1)); pinned against the O(N^2) evaluation in the tests.   */
/* ------------------------------------------------------------------------ */
static void ntt_fwd(const or_ctx* c, int pi, u64* a) {
    int N = c->n;
    u64 q = c->p[pi];
    const u64* w = c->psi_rev[pi];
    int t = N;
    for (int m = 1; m < N; m <<= 1) {
        t >>= 1;
        for (int i = 0; i < m; i++) {
            int j1 = 2 * i * t;
            u64 S = w[m + i];
            for (int j = j1; j < j1 + t; j++) {
                u64 U = a[j], V = mmul(a[j + t], S, q);
                a[j] = madd(U, V, q);
                a[j + t] = msub(U, V, q);
            }
        }
    }
}

static void ntt_inv(const or_ctx* c, int pi, u64* a) {
    int N = c->n;
    u64 q = c->p[pi];
    const u64* w = c->ipsi_rev[pi];
    int t = 1;
    for (int m = N >> 1; m >= 1; m >>= 1) {
        int j1 = 0;
        for (int i = 0; i < m; i++) {
            u64 S = w[m + i];
            for (int j = j1; j < j1 + t; j++) {
                u64 U = a[j], V = a[j + t];
                a[j] = madd(U, V, q);
                a[j + t] = mmul(msub(U, V, q), S, q);
            }
            j1 += 2 * t;
        }
        t <<= 1;
    }
    for (int j = 0; j < N; j++) a[j] = mmul(a[j], c->ninv[pi], q);
}

void or_ntt_fwd(const or_ctx* c, int pi, u64* a) { ntt_fwd(c, pi, a); }
void or_ntt_inv(const or_ctx* c, int pi, u64* a) { ntt_inv(c, pi, a); }

/* ------------------------------------------------------------------------ */
/* Automorphism sigma_g: a(X) -> a(X^g), g odd (Section "Hoisting and double */
/* hoisting": a rotation is a Galois automorphism then a key switch).        */
/* ------------------------------------------------------------------------ */
static void automorph_coef(const or_ctx* c, u64 g, u64 q, const u64* in, u64* out) {
    u64 N = (u64)c->n, M = 2 * N;
    for (u64 j = 0; j < N; j++) {
        u64 e = (j * g) % M;
        if (e < N) out[e] = in[j];
        else out[e - N] = (q - in[j]) % q;
    }
}

/* same map in evaluation form: value at psi^e of sigma_g(a) is a(psi^(e g)) */
static void automorph_eval(const or_ctx* c, u64 g, const u64* in, u64* out) {
    int N = c->n, L = c->log_n;
    u64 M = 2 * (u64)N;
    for (int k = 0; k < N; k++) {
        u64 e = 2 * (u64)brev((u32)k, L) + 1;
        u64 e2 = (e * g) % M;
        u32 k2 = brev((u32)((e2 - 1) / 2), L);
        out[k] = in[k2];
    }
}

void or_automorph_coef(const or_ctx* c, u64 g, int pi, const u64* in, u64* out) {
    automorph_coef(c, g, c->p[pi], in, out);
}
void or_automorph_eval(const or_ctx* c, u64 g, const u64* in, u64* out) { automorph_eval(c, g, in, out); }

/* Galois element of a left rotation by k slots (reading R4): 5^k mod 2N. */
u64 or_galois(const or_ctx* c, long k) {
    long n = c->n / 2;
    long kk = ((k % n) + n) % n;
    return mpow(5, (u64)kk, 2 * (u64)c->n);
}

/* ------------------------------------------------------------------------ */
/* ChaCha20 block function (RFC 8439, Section 2.3) and the samplers built on */
/* it (reading R6). One stream per sampled object: key = (seed, constant),   */
/* nonce = (object id lo, object id hi, limb), counter from 0.              */
/* ------------------------------------------------------------------------ */
#define ROTL32(v, n) (((v) << (n)) | ((v) >> (32 - (n))))
#define QR(a, b, c, d)                                                                    \
    a += b; d ^= a; d = ROTL32(d, 16);                                                   \
    c += d; b ^= c; b = ROTL32(b, 12);                                                   \
    a += b; d ^= a; d = ROTL32(d, 8);                                                    \
    c += d; b ^= c; b = ROTL32(b, 7);

void or_chacha20_block(const u32 key[8], u32 counter, const u32 nonce[3], uint8_t out[64]) {
    u32 st[16], x[16];
    st[0] = 0x61707865u; st[1] = 0x3320646eu; st[2] = 0x79622d32u; st[3] = 0x6b206574u;
    for (int i = 0; i < 8; i++) st[4 + i] = key[i];
    st[12] = counter;
    st[13] = nonce[0]; st[14] = nonce[1]; st[15] = nonce[2];
    memcpy(x, st, sizeof(st));
    for (int r = 0; r < 10; r++) {
        QR(x[0], x[4], x[8], x[12]);
        QR(x[1], x[5], x[9], x[13]);
        QR(x[2], x[6], x[10], x[14]);
        QR(x[3], x[7], x[11], x[15]);
        QR(x[0], x[5], x[10], x[15]);
        QR(x[1], x[6], x[11], x[12]);
        QR(x[2], x[7], x[8], x[13]);
        QR(x[3], x[4], x[9], x[14]);
    }
    for (int i = 0; i < 16; i++) {
        u32 v = x[i] + st[i];
        out[4 * i + 0] = (uint8_t)(v);
        out[4 * i + 1] = (uint8_t)(v >> 8);
        out[4 * i + 2] = (uint8_t)(v >> 16);
        out[4 * i + 3] = (uint8_t)(v >> 24);
    }
}

typedef struct {
    u32 key[8], nonce[3], ctr;
    uint8_t buf[64];
    int pos;
} prng_t;

static void prng_init(prng_t* g, u64 seed, u64 obj, u32 limb) {
    g->key[0] = (u32)seed;
    g->key[1] = (u32)(seed >> 32);
    g->key[2] = 0x2d726601u; /* fixed key words: "\x01fr-" */
    for (int i = 3; i < 8; i++) g->key[i] = 0;
    g->nonce[0] = (u32)obj;
    g->nonce[1] = (u32)(obj >> 32);
    g->nonce[2] = limb;
    g->ctr = 0;
    g->pos = 64;
}
static uint8_t prng_byte(prng_t* g) {
    if (g->pos == 64) {
        or_chacha20_block(g->key, g->ctr, g->nonce, g->buf);
        g->ctr++;
        g->pos = 0;
    }
    return g->buf[g->pos++];
}
static u64 prng_bytes_le(prng_t* g, int nb) {
    u64 v = 0;
    for (int i = 0; i < nb; i++) v |= (u64)prng_byte(g) << (8 * i);
    return v;
}

/* uniform ternary {-1,0,1}: byte b < 255 accepted, value b mod 3 - 1 */
static void sample_ternary(u64 seed, u64 obj, int n, int8_t* out) {
    prng_t g;
    prng_init(&g, seed, obj, 0);
    for (int i = 0; i < n; i++) {
        uint8_t b;
        do { b = prng_byte(&g); } while (b == 255);
        out[i] = (int8_t)((int)(b % 3) - 1);
    }
}
/* centered binomial, eta = 21: 6 bytes, popcount(bits 0..20) - popcount(bits 21..41) */
static void sample_cbd(u64 seed, u64 obj, int n, int32_t* out) {
    prng_t g;
    prng_init(&g, seed, obj, 0);
    for (int i = 0; i < n; i++) {
        u64 x = prng_bytes_le(&g, 6);
        out[i] = __builtin_popcountll(x & 0x1FFFFFull) - __builtin_popcountll((x >> 21) & 0x1FFFFFull);
    }
}
/* uniform mod q: 8-byte little-endian word masked to bitlen(q), rejected if >= q */
static void sample_uniform(u64 seed, u64 obj, u32 limb, u64 q, int n, u64* out) {
    prng_t g;
    prng_init(&g, seed, obj, limb);
    int bl = 64 - __builtin_clzll(q);
    u64 mask = (bl == 64) ? ~(u64)0 : (((u64)1 << bl) - 1);
    for (int i = 0; i < n; i++) {
        u64 v;
        do { v = prng_bytes_le(&g, 8) & mask; } while (v >= q);
        out[i] = v;
    }
}

void or_sample_ternary(u64 seed, u64 obj, int n, int8_t* out) { sample_ternary(seed, obj, n, out); }
void or_sample_cbd(u64 seed, u64 obj, int n, int32_t* out) { sample_cbd(seed, obj, n, out); }
void or_sample_uniform(u64 seed, u64 obj, u32 limb, u64 q, int n, u64* out) {
    sample_uniform(seed, obj, limb, q, n, out);
}

/* object ids of the sampled objects */
#define OBJ_S 0x01ull
#define OBJ_PK_A 0x02ull
#define OBJ_PK_E 0x03ull
#define OBJ_ENC_V 0x11ull
#define OBJ_ENC_E0 0x12ull
#define OBJ_ENC_E1 0x13ull
static u64 obj_evk(int relin, u64 g, int d, int which) {
    return ((u64)(relin ? 2 : 1) << 40) | (g << 8) | ((u64)d << 1) | (u64)which;
}

/* ------------------------------------------------------------------------ */
/* Encoding (Section "CKKS", encoding paragraph; reading R5): inverse special */
/* FFT over the 5^j slot order, scale by Delta, round half away from zero.   */
/* ------------------------------------------------------------------------ */
static void bitrev_cplx(double* re, double* im, int n) {
    int lg = 0;
    while ((1 << lg) < n) lg++;
    for (int i = 0; i < n; i++) {
        int j = (int)brev((u32)i, lg);
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
}

/* w = inverse special DFT of z (times n, the 1/n is applied by the caller):
 * w_c = sum_j z_j zeta^(-5^j c); stages len = n..2, then bit reversal. */
static void fft_special_inv(const or_ctx* c, double* re, double* im) {
    int n = c->n / 2;
    u64 M = 2 * (u64)c->n;
    for (int len = n; len >= 2; len >>= 1) {
        int lenh = len >> 1;
        u64 lenq = (u64)len << 2;
        u64 gap = M / lenq;
        for (int i = 0; i < n; i += len) {
            for (int j = 0; j < lenh; j++) {
                u64 idx = (lenq - (c->rot_group[j] % lenq)) * gap;
                double ar = re[i + j], ai = im[i + j];
                double br = re[i + j + lenh], bi = im[i + j + lenh];
                double ur = ar + br, ui = ai + bi;
                double vr = ar - br, vi = ai - bi;
                double wr = c->zr[idx], wi = c->zi[idx];
                re[i + j] = ur;
                im[i + j] = ui;
                re[i + j + lenh] = vr * wr - vi * wi;
                im[i + j + lenh] = vr * wi + vi * wr;
            }
        }
    }
    bitrev_cplx(re, im, n);
}

/* forward special DFT: z_j = sum_c w_c zeta^(5^j c) */
static void fft_special_fwd(const or_ctx* c, double* re, double* im) {
    int n = c->n / 2;
    u64 M = 2 * (u64)c->n;
    bitrev_cplx(re, im, n);
    for (int len = 2; len <= n; len <<= 1) {
        int lenh = len >> 1;
        u64 lenq = (u64)len << 2;
        u64 gap = M / lenq;
        for (int i = 0; i < n; i += len) {
            for (int j = 0; j < lenh; j++) {
                u64 idx = (c->rot_group[j] % lenq) * gap;
                double ar = re[i + j], ai = im[i + j];
                double br = re[i + j + lenh], bi = im[i + j + lenh];
                double wr = c->zr[idx], wi = c->zi[idx];
                double vr = br * wr - bi * wi;
                double vi = br * wi + bi * wr;
                re[i + j] = ar + vr;
                im[i + j] = ai + vi;
                re[i + j + lenh] = ar - vr;
                im[i + j + lenh] = ai - vi;
            }
        }
    }
}

/* integer coefficients of encode(z) at scale 2^scale_bits: z real, n = N/2 slots */
void or_encode_coeffs(const or_ctx* c, const double* z, int scale_bits, int64_t* m) {
    int n = c->n / 2;
    double* re = (double*)malloc(sizeof(double) * n);
    double* im = (double*)malloc(sizeof(double) * n);
    for (int j = 0; j < n; j++) { re[j] = z[j]; im[j] = 0.0; }
    fft_special_inv(c, re, im);
    double inv_n = 1.0 / (double)n;
    double delta = ldexp(1.0, scale_bits);
    for (int k = 0; k < n; k++) {
        m[k] = llround((re[k] * inv_n) * delta);
        m[k + n] = llround((im[k] * inv_n) * delta);
    }
    free(re);
    free(im);
}

/* residues [level+1][N] (coefficient form) of encode(z) */
void or_encode(const or_ctx* c, const double* z, int level, int scale_bits, u64* out) {
    int N = c->n;
    int64_t* m = (int64_t*)malloc(sizeof(int64_t) * N);
    or_encode_coeffs(c, z, scale_bits, m);
    for (int i = 0; i <= level; i++)
        for (int k = 0; k < N; k++) out[(size_t)i * N + k] = mred_s(m[k], c->p[i]);
    free(m);
}

/* decode of coefficients x (length N): z_j = Re m(zeta^(5^j)) / scale */
static void decode_values(const or_ctx* c, const double* x, double scale, double* z) {
    int n = c->n / 2;
    double* re = (double*)malloc(sizeof(double) * n);
    double* im = (double*)malloc(sizeof(double) * n);
    for (int k = 0; k < n; k++) { re[k] = x[k]; im[k] = x[k + n]; }
    fft_special_fwd(c, re, im);
    for (int j = 0; j < n; j++) z[j] = re[j] / scale;
    free(re);
    free(im);
}

void or_decode_coeffs(const or_ctx* c, const int64_t* x, double scale, double* z) {
    double* v = (double*)malloc(sizeof(double) * c->n);
    for (int k = 0; k < c->n; k++) v[k] = (double)x[k];
    decode_values(c, v, scale, z);
    free(v);
}

/* ------------------------------------------------------------------------ */
/* Ring products through the NTT                                             */
/* ------------------------------------------------------------------------ */
/* out = a*b in R_{p_pi}, all in coefficient form */
static void ring_mul(const or_ctx* c, int pi, const u64* a, const u64* b, u64* out) {
    int N = c->n;
    u64 q = c->p[pi];
    u64* A = (u64*)malloc(sizeof(u64) * N);
    u64* B = (u64*)malloc(sizeof(u64) * N);
    memcpy(A, a, sizeof(u64) * N);
    memcpy(B, b, sizeof(u64) * N);
    ntt_fwd(c, pi, A);
    ntt_fwd(c, pi, B);
    for (int k = 0; k < N; k++) A[k] = mmul(A[k], B[k], q);
    ntt_inv(c, pi, A);
    memcpy(out, A, sizeof(u64) * N);
    free(A);
    free(B);
}

/* ------------------------------------------------------------------------ */
/* Keys (Section "CKKS": RLWE public key; reading R6)                        */
/*   pk = (-a s + e, a) over Q; a sampled in evaluation form.                 */
/*   hybrid key-switching key for s' (digit d with limbs D_d, alpha per digit)*/
/*   evk_d = (-a_d s + e_d + [P]_{q_i} s' on i in D_d, a_d) over Q u P.       */
/* ------------------------------------------------------------------------ */
static int ntot(const or_ctx* c) { return c->nq + c->np; }
static int beta_top(const or_ctx* c) { return c->ndig; }
/* digits at level l: those with dstart[d] <= l, truncated to [0, l] */
static int beta_at(const or_ctx* c, int l) {
    int b = 0;
    while (b < c->ndig && c->dstart[b] <= l) b++;
    return b;
}
static void digit_range(const or_ctx* c, int l, int d, int* lo, int* hi) {
    *lo = c->dstart[d];
    *hi = c->dstart[d + 1] < l + 1 ? c->dstart[d + 1] : l + 1;
}
int or_ndig(const or_ctx* c) { return c->ndig; }
int or_dstart(const or_ctx* c, int d) { return c->dstart[d]; }

or_keys* or_keygen(const or_ctx* c, u64 seed) {
    int N = c->n, T = ntot(c);
    or_keys* k = (or_keys*)calloc(1, sizeof(or_keys));
    k->seed = seed;
    k->s = (int8_t*)malloc(N);
    sample_ternary(seed, OBJ_S, N, k->s);
    k->s_eval = (u64*)malloc(sizeof(u64) * (size_t)T * N);
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < T; i++) {
        u64* r = k->s_eval + (size_t)i * N;
        for (int j = 0; j < N; j++) r[j] = mred_s(k->s[j], c->p[i]);
        ntt_fwd(c, i, r);
    }
    k->pk0 = (u64*)malloc(sizeof(u64) * (size_t)c->nq * N);
    k->pk1 = (u64*)malloc(sizeof(u64) * (size_t)c->nq * N);
    int32_t* e = (int32_t*)malloc(sizeof(int32_t) * N);
    sample_cbd(seed, OBJ_PK_E, N, e);
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < c->nq; i++) {
        u64 q = c->p[i];
        u64* a = k->pk1 + (size_t)i * N;
        u64* b = k->pk0 + (size_t)i * N;
        sample_uniform(seed, OBJ_PK_A, (u32)i, q, N, a);
        for (int j = 0; j < N; j++) b[j] = mred_s(e[j], q);
        ntt_fwd(c, i, b);
        for (int j = 0; j < N; j++) b[j] = msub(b[j], mmul(a[j], k->s_eval[(size_t)i * N + j], q), q);
    }
    free(e);
    return k;
}

void or_free_keys(or_keys* k) {
    if (!k) return;
    free(k->s); free(k->s_eval); free(k->pk0); free(k->pk1); free(k->relin);
    free(k);
}

void or_secret(const or_keys* k, int n, int8_t* out) { memcpy(out, k->s, n); }

/* evk for s' = sigma_g(s) (relin == 0) or s^2 (relin == 1); out [beta][2][T][N] eval form */
void or_make_evk(const or_ctx* c, const or_keys* k, int relin, u64 g, u64* out) {
    int N = c->n, T = ntot(c), beta = beta_top(c);
    u64 P_mod[OR_MAXP];
    for (int i = 0; i < T; i++) {
        u64 q = c->p[i];
        u64 pm = 1 % q;
        for (int j = 0; j < c->np; j++) pm = mmul(pm, c->p[c->nq + j] % q, q);
        P_mod[i] = pm;
    }
    for (int d = 0; d < beta; d++) {
        int lo = c->dstart[d], hi = c->dstart[d + 1];
        int32_t* e = (int32_t*)malloc(sizeof(int32_t) * N);
        sample_cbd(k->seed, obj_evk(relin, relin ? 0 : g, d, 1), N, e);
#pragma omp parallel for schedule(dynamic)
        for (int i = 0; i < T; i++) {
            u64 q = c->p[i];
            u64* b = out + (((size_t)d * 2 + 0) * T + i) * N;
            u64* a = out + (((size_t)d * 2 + 1) * T + i) * N;
            const u64* se = k->s_eval + (size_t)i * N;
            sample_uniform(k->seed, obj_evk(relin, relin ? 0 : g, d, 0), (u32)i, q, N, a);
            for (int j = 0; j < N; j++) b[j] = mred_s(e[j], q);
            ntt_fwd(c, i, b);
            u64* sp = (u64*)malloc(sizeof(u64) * N);
            if (relin) {
                for (int j = 0; j < N; j++) sp[j] = mmul(se[j], se[j], q);
            } else {
                automorph_eval(c, g, se, sp);
            }
            int in_digit = (i >= lo && i < hi);
            for (int j = 0; j < N; j++) {
                u64 v = msub(b[j], mmul(a[j], se[j], q), q);
                if (in_digit) v = madd(v, mmul(P_mod[i], sp[j], q), q);
                b[j] = v;
            }
            free(sp);
        }
        free(e);
    }
}

/* ------------------------------------------------------------------------ */
/* Encryption / decryption (Section "CKKS", encryption paragraph)            */
/* ------------------------------------------------------------------------ */
/* out: [2][nq][N] coefficient form, level nq-1; z has n = N/2 real slots */
void or_encrypt(const or_ctx* c, const or_keys* k, const double* z, u64 seed, u64* out) {
    int N = c->n, L = c->nq - 1;
    u64* m = (u64*)malloc(sizeof(u64) * (size_t)c->nq * N);
    or_encode(c, z, L, c->scale_bits, m);
    int8_t* v = (int8_t*)malloc(N);
    int32_t* e0 = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* e1 = (int32_t*)malloc(sizeof(int32_t) * N);
    sample_ternary(seed, OBJ_ENC_V, N, v);
    sample_cbd(seed, OBJ_ENC_E0, N, e0);
    sample_cbd(seed, OBJ_ENC_E1, N, e1);
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < c->nq; i++) {
        u64 q = c->p[i];
        u64* V = (u64*)malloc(sizeof(u64) * N);
        u64* c0 = out + (size_t)i * N;
        u64* c1 = out + ((size_t)c->nq + i) * N;
        for (int j = 0; j < N; j++) V[j] = mred_s(v[j], q);
        ntt_fwd(c, i, V);
        for (int j = 0; j < N; j++) {
            c0[j] = mmul(V[j], k->pk0[(size_t)i * N + j], q);
            c1[j] = mmul(V[j], k->pk1[(size_t)i * N + j], q);
        }
        ntt_inv(c, i, c0);
        ntt_inv(c, i, c1);
        for (int j = 0; j < N; j++) {
            c0[j] = madd(madd(c0[j], mred_s(e0[j], q), q), m[(size_t)i * N + j], q);
            c1[j] = madd(c1[j], mred_s(e1[j], q), q);
        }
        free(V);
    }
    free(m); free(v); free(e0); free(e1);
}

/* m = c0 + c1 s on limb 0 (q0 is 60-bit, |m| << q0/2), centered */
void or_decrypt_coeffs(const or_ctx* c, const or_keys* k, const u64* ct, int level, int64_t* x) {
    int N = c->n;
    u64 q = c->p[0];
    const u64* c0 = ct;
    const u64* c1 = ct + (size_t)(level + 1) * N;
    u64* s0 = (u64*)malloc(sizeof(u64) * N);
    u64* t = (u64*)malloc(sizeof(u64) * N);
    for (int j = 0; j < N; j++) s0[j] = mred_s(k->s[j], q);
    ring_mul(c, 0, c1, s0, t);
    for (int j = 0; j < N; j++) {
        u64 v = madd(t[j], c0[j], q);
        x[j] = (v > (q - 1) / 2) ? -(int64_t)(q - v) : (int64_t)v;
    }
    free(s0);
    free(t);
}

/* m = c0 + c1 s as real numbers: centered CRT of limbs 0 and 1 when level >= 1
 * (|m| < q0 q1 / 2), limb 0 alone at level 0. */
void or_decrypt_values(const or_ctx* c, const or_keys* k, const u64* ct, int level, double* x) {
    int N = c->n;
    int nl = level >= 1 ? 2 : 1;
    u64* v[2];
    for (int i = 0; i < nl; i++) {
        u64 q = c->p[i];
        const u64* c0 = ct + (size_t)i * N;
        const u64* c1 = ct + (size_t)(level + 1 + i) * N;
        u64* s0 = (u64*)malloc(sizeof(u64) * N);
        v[i] = (u64*)malloc(sizeof(u64) * N);
        for (int j = 0; j < N; j++) s0[j] = mred_s(k->s[j], q);
        ring_mul(c, i, c1, s0, v[i]);
        for (int j = 0; j < N; j++) v[i][j] = madd(v[i][j], c0[j], q);
        free(s0);
    }
    if (nl == 1) {
        u64 q = c->p[0];
        for (int j = 0; j < N; j++) x[j] = (v[0][j] > (q - 1) / 2) ? -(double)(q - v[0][j]) : (double)v[0][j];
        free(v[0]);
        return;
    }
    u64 q0 = c->p[0], q1 = c->p[1];
    u64 q0inv = minv(q0 % q1, q1);
    u128 Q = (u128)q0 * q1;
    for (int j = 0; j < N; j++) {
        u64 h = mmul(msub(v[1][j], v[0][j] % q1, q1), q0inv, q1);
        u128 y = (u128)v[0][j] + (u128)q0 * h;   /* in [0, q0 q1) */
        if (y > (Q - 1) / 2) x[j] = -(double)(Q - y);
        else x[j] = (double)y;
    }
    free(v[0]);
    free(v[1]);
}

static void decode_values(const or_ctx* c, const double* x, double scale, double* z);

void or_decrypt(const or_ctx* c, const or_keys* k, const u64* ct, int level, double scale, double* z) {
    double* x = (double*)malloc(sizeof(double) * c->n);
    or_decrypt_values(c, k, ct, level, x);
    decode_values(c, x, scale, z);
    free(x);
}

/* ------------------------------------------------------------------------ */
/* Key switching (Section "Hoisting and double hoisting"; reading R6b)        */
/*   ModUp: per digit D_d, fast base conversion of [c]_{D_d} to every other  */
/*   limb of Q_l u P, then NTT. The automorphism is applied AFTER ModUp.     */
/*   IP: sum_d ext_d (.) evk_d. ModDown: (x - FastBConv_{P->Q}(x mod P))/P.  */
/* ------------------------------------------------------------------------ */
/* FastBConv of residues x[i] (basis src[0..ns)) to modulus t:
 * sum_i [x_i * (B/b_i)^-1]_{b_i} * [B/b_i]_t  mod t */
static void bconv_consts(const or_ctx* c, const int* src, int ns, u64 t, u64* inv_hat, u64* hat_t) {
    for (int i = 0; i < ns; i++) {
        u64 bi = c->p[src[i]];
        u64 h = 1 % bi, ht = 1 % t;
        for (int j = 0; j < ns; j++) {
            if (j == i) continue;
            h = mmul(h, c->p[src[j]] % bi, bi);
            ht = mmul(ht, c->p[src[j]] % t, t);
        }
        inv_hat[i] = minv(h, bi);
        hat_t[i] = ht;
    }
}

/* limb (prime) index of position pos at level l in the extended basis Q_l u P */
static int ext_limb(const or_ctx* c, int l, int pos) { return pos <= l ? pos : c->nq + (pos - (l + 1)); }

/* ModUp of coefficient-form c1 [l+1][N] into ext [beta_l][npos][N], evaluation form */
static void modup(const or_ctx* c, const u64* a, int l, u64* ext) {
    int N = c->n, npos = l + 1 + c->np;
    int beta = beta_at(c, l);
    for (int d = 0; d < beta; d++) {
        int lo, hi;
        digit_range(c, l, d, &lo, &hi);
        int ns = hi - lo;
        int src[OR_MAXP];
        for (int i = 0; i < ns; i++) src[i] = lo + i;
#pragma omp parallel for schedule(dynamic)
        for (int pos = 0; pos < npos; pos++) {
            int li = ext_limb(c, l, pos);
            u64 t = c->p[li];
            u64* out = ext + ((size_t)d * npos + pos) * N;
            if (pos >= lo && pos < hi) {
                memcpy(out, a + (size_t)pos * N, sizeof(u64) * N);
            } else {
                u64 inv_hat[OR_MAXP], hat_t[OR_MAXP];
                bconv_consts(c, src, ns, t, inv_hat, hat_t);
                for (int j = 0; j < N; j++) {
                    u64 acc = 0;
                    for (int i = 0; i < ns; i++) {
                        u64 bi = c->p[src[i]];
                        u64 y = mmul(a[(size_t)src[i] * N + j], inv_hat[i], bi);
                        acc = madd(acc, mmul(y % t, hat_t[i], t), t);
                    }
                    out[j] = acc;
                }
            }
            ntt_fwd(c, li, out);
        }
    }
}

/* ModDown of acc [npos][N] (evaluation form) into out [l+1][N] coefficient form */
static void moddown(const or_ctx* c, u64* acc, int l, u64* out) {
    int N = c->n, npos = l + 1 + c->np;
#pragma omp parallel for schedule(dynamic)
    for (int pos = 0; pos < npos; pos++) ntt_inv(c, ext_limb(c, l, pos), acc + (size_t)pos * N);
    int src[OR_MAXP];
    for (int j = 0; j < c->np; j++) src[j] = c->nq + j;
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i <= l; i++) {
        u64 q = c->p[i];
        u64 inv_hat[OR_MAXP], hat_t[OR_MAXP];
        bconv_consts(c, src, c->np, q, inv_hat, hat_t);
        u64 Pm = 1 % q;
        for (int j = 0; j < c->np; j++) Pm = mmul(Pm, c->p[c->nq + j] % q, q);
        u64 Pinv = minv(Pm, q);
        for (int k = 0; k < N; k++) {
            u64 conv = 0;
            for (int j = 0; j < c->np; j++) {
                u64 pj = c->p[c->nq + j];
                u64 y = mmul(acc[((size_t)(l + 1 + j)) * N + k], inv_hat[j], pj);
                conv = madd(conv, mmul(y % q, hat_t[j], q), q);
            }
            out[(size_t)i * N + k] = mmul(msub(acc[(size_t)i * N + k], conv, q), Pinv, q);
        }
    }
}

/* inner product of ext (shared ModUp) with one key, automorphism g applied to ext */
static void keyswitch_ip(const or_ctx* c, const u64* ext, int l, const u64* evk, u64 g, u64* acc0, u64* acc1) {
    int N = c->n, T = ntot(c), npos = l + 1 + c->np;
    int beta = beta_at(c, l);
#pragma omp parallel for schedule(dynamic)
    for (int pos = 0; pos < npos; pos++) {
        int li = ext_limb(c, l, pos);
        u64 q = c->p[li];
        u64* r0 = acc0 + (size_t)pos * N;
        u64* r1 = acc1 + (size_t)pos * N;
        u64* tmp = (u64*)malloc(sizeof(u64) * N);
        memset(r0, 0, sizeof(u64) * N);
        memset(r1, 0, sizeof(u64) * N);
        for (int d = 0; d < beta; d++) {
            const u64* e = ext + ((size_t)d * npos + pos) * N;
            if (g != 1) automorph_eval(c, g, e, tmp);
            else memcpy(tmp, e, sizeof(u64) * N);
            const u64* k0 = evk + (((size_t)d * 2 + 0) * T + li) * N;
            const u64* k1 = evk + (((size_t)d * 2 + 1) * T + li) * N;
            for (int j = 0; j < N; j++) {
                r0[j] = madd(r0[j], mmul(tmp[j], k0[j], q), q);
                r1[j] = madd(r1[j], mmul(tmp[j], k1[j], q), q);
            }
        }
        free(tmp);
    }
}

static size_t evk_words(const or_ctx* c) { return (size_t)beta_top(c) * 2 * ntot(c) * c->n; }

/* Hoisted rotations (Algorithm 1, step 1: one ModUp shared by every rotation).
 * ct at level l (coefficient form, [2][l+1][N]); out: nr cts in the same layout. */
void or_hoisted_rotate(const or_ctx* c, const or_keys* k, const u64* ct, int l, const long* rots, int nr,
                       u64* out) {
    int N = c->n, npos = l + 1 + c->np;
    int beta = beta_at(c, l);
    size_t ctw = (size_t)2 * (l + 1) * N;
    u64* ext = (u64*)malloc(sizeof(u64) * (size_t)beta * npos * N);
    modup(c, ct + (size_t)(l + 1) * N, l, ext);
    u64* evk = (u64*)malloc(sizeof(u64) * evk_words(c));
    u64* acc0 = (u64*)malloc(sizeof(u64) * (size_t)npos * N);
    u64* acc1 = (u64*)malloc(sizeof(u64) * (size_t)npos * N);
    for (int r = 0; r < nr; r++) {
        u64 g = or_galois(c, rots[r]);
        u64* o = out + (size_t)r * ctw;
        if (g == 1) { memcpy(o, ct, sizeof(u64) * ctw); continue; }
        or_make_evk(c, k, 0, g, evk);
        keyswitch_ip(c, ext, l, evk, g, acc0, acc1);
        moddown(c, acc0, l, o);
        moddown(c, acc1, l, o + (size_t)(l + 1) * N);
        for (int i = 0; i <= l; i++) {
            u64 q = c->p[i];
            u64* t = (u64*)malloc(sizeof(u64) * N);
            automorph_coef(c, g, q, ct + (size_t)i * N, t);
            for (int j = 0; j < N; j++) o[(size_t)i * N + j] = madd(o[(size_t)i * N + j], t[j], q);
            free(t);
        }
    }
    free(ext); free(evk); free(acc0); free(acc1);
}

void or_rotate(const or_ctx* c, const or_keys* k, const u64* ct, int l, long rot, u64* out) {
    or_hoisted_rotate(c, k, ct, l, &rot, 1, out);
}

/* ------------------------------------------------------------------------ */
/* Rescale (Section "CKKS", multiplication paragraph; reading R8): divide by  */
/* q_l with the centered lift of the last limb, drop it.                     */
/* ------------------------------------------------------------------------ */
void or_rescale(const or_ctx* c, const u64* ct, int l, u64* out) {
    int N = c->n;
    u64 ql = c->p[l];
    for (int t = 0; t < 2; t++) {
        const u64* in = ct + (size_t)t * (l + 1) * N;
        u64* o = out + (size_t)t * l * N;
        for (int i = 0; i < l; i++) {
            u64 q = c->p[i];
            u64 inv = minv(ql % q, q);
            for (int j = 0; j < N; j++) {
                u64 x = in[(size_t)l * N + j];
                int64_t v = (x > (ql - 1) / 2) ? -(int64_t)(ql - x) : (int64_t)x;
                o[(size_t)i * N + j] = mmul(msub(in[(size_t)i * N + j], mred_s(v, q), q), inv, q);
            }
        }
    }
}

/* drop limbs: level l -> l2 < l */
void or_drop(const or_ctx* c, const u64* ct, int l, int l2, u64* out) {
    int N = c->n;
    memmove(out, ct, sizeof(u64) * (size_t)(l2 + 1) * N);
    memmove(out + (size_t)(l2 + 1) * N, ct + (size_t)(l + 1) * N, sizeof(u64) * (size_t)(l2 + 1) * N);
}

void or_add(const or_ctx* c, const u64* a, const u64* b, int l, u64* out) {
    int N = c->n;
    for (int t = 0; t < 2; t++)
        for (int i = 0; i <= l; i++)
            for (int j = 0; j < N; j++) {
                size_t o = ((size_t)t * (l + 1) + i) * N + j;
                out[o] = madd(a[o], b[o], c->p[i]);
            }
}

/* ------------------------------------------------------------------------ */
/* Ciphertext product + relinearisation (Section "CKKS", multiplication)     */
/*   (d0,d1,d2) = (a0 b0, a0 b1 + a1 b0, a1 b1); out = (d0,d1) + KS_{s^2}(d2) */
/* ------------------------------------------------------------------------ */
static const u64* relin_key(const or_ctx* c, or_keys* k) {
    if (!k->relin) {
        k->relin = (u64*)malloc(sizeof(u64) * evk_words(c));
        or_make_evk(c, k, 1, 0, k->relin);
    }
    return k->relin;
}

/* out (a ct [2][l+1][N], coefficient form) += KS_{s^2}(d2): the relinearisation of (d0,d1,d2)
 * with (d0,d1) already in out */
static void relin_add(const or_ctx* c, or_keys* k, const u64* d2, int l, u64* out) {
    int N = c->n, npos = l + 1 + c->np;
    int beta = beta_at(c, l);
    const u64* rk = relin_key(c, k);
    u64* ext = (u64*)malloc(sizeof(u64) * (size_t)beta * npos * N);
    u64* acc0 = (u64*)malloc(sizeof(u64) * (size_t)npos * N);
    u64* acc1 = (u64*)malloc(sizeof(u64) * (size_t)npos * N);
    u64* ks = (u64*)malloc(sizeof(u64) * (size_t)2 * (l + 1) * N);
    modup(c, d2, l, ext);
    keyswitch_ip(c, ext, l, rk, 1, acc0, acc1);
    moddown(c, acc0, l, ks);
    moddown(c, acc1, l, ks + (size_t)(l + 1) * N);
    or_add(c, out, ks, l, out);
    free(ext); free(acc0); free(acc1); free(ks);
}

void or_mul_relin(const or_ctx* c, or_keys* k, const u64* a, const u64* b, int l, u64* out) {
    int N = c->n;
    u64* d2 = (u64*)malloc(sizeof(u64) * (size_t)(l + 1) * N);
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i <= l; i++) {
        u64 q = c->p[i];
        u64* A0 = (u64*)malloc(sizeof(u64) * N); u64* A1 = (u64*)malloc(sizeof(u64) * N);
        u64* B0 = (u64*)malloc(sizeof(u64) * N); u64* B1 = (u64*)malloc(sizeof(u64) * N);
        memcpy(A0, a + (size_t)i * N, sizeof(u64) * N);
        memcpy(A1, a + (size_t)(l + 1 + i) * N, sizeof(u64) * N);
        memcpy(B0, b + (size_t)i * N, sizeof(u64) * N);
        memcpy(B1, b + (size_t)(l + 1 + i) * N, sizeof(u64) * N);
        ntt_fwd(c, i, A0); ntt_fwd(c, i, A1); ntt_fwd(c, i, B0); ntt_fwd(c, i, B1);
        u64* o0 = out + (size_t)i * N;
        u64* o1 = out + (size_t)(l + 1 + i) * N;
        u64* o2 = d2 + (size_t)i * N;
        for (int j = 0; j < N; j++) {
            o0[j] = mmul(A0[j], B0[j], q);
            o1[j] = madd(mmul(A0[j], B1[j], q), mmul(A1[j], B0[j], q), q);
            o2[j] = mmul(A1[j], B1[j], q);
        }
        ntt_inv(c, i, o0); ntt_inv(c, i, o1); ntt_inv(c, i, o2);
        free(A0); free(A1); free(B0); free(B1);
    }
    relin_add(c, k, d2, l, out);
    free(d2);
}

/* ------------------------------------------------------------------------ */
/* Scalar operations used by the Chebyshev evaluator                         */
/* ------------------------------------------------------------------------ */
/* ct * v (v a signed integer), coefficient-wise */
static void mul_int(const or_ctx* c, u64* ct, int l, int64_t v) {
    int N = c->n;
    for (int t = 0; t < 2; t++)
        for (int i = 0; i <= l; i++) {
            u64 q = c->p[i], r = mred_s(v, q);
            u64* x = ct + ((size_t)t * (l + 1) + i) * N;
            for (int j = 0; j < N; j++) x[j] = mmul(x[j], r, q);
        }
}
/* c0 += v (a constant polynomial, v given by its residues through vr(q)) */
static void add_const_res(const or_ctx* c, u64* ct, int l, int64_t v, int times_delta) {
    int N = c->n;
    for (int i = 0; i <= l; i++) {
        u64 q = c->p[i];
        u64 r = mred_s(v, q);
        if (times_delta) r = mmul(r, mpow(2, (u64)c->scale_bits, q), q);
        ct[(size_t)i * N + 0] = madd(ct[(size_t)i * N + 0], r, q);
    }
    (void)N;
}

/* ------------------------------------------------------------------------ */
/* Chebyshev threshold (Section "GPU-native Chebyshev comparison", Eq.       */
/* eq:cheb-sign; reading R9): interpolant of step(x - tau) at the n+1        */
/* Chebyshev nodes, evaluated by Paterson-Stockmeyer with d1 = 2 and the     */
/* Chebyshev division p = q T_M + r.                                         */
/* ------------------------------------------------------------------------ */
/* interpolant of f(x) = 1 for x >= tau, `low` below (low = 0: step(x - tau); low = -1:
 * sign(x - tau), the input of the hybrid comparator) */
void or_cheb_coeffs_lo(int n, double tau, double low, double* cf) {
    for (int k = 0; k <= n; k++) {
        double s = 0.0;
        for (int j = 0; j <= n; j++) {
            double theta = M_PI * ((double)j + 0.5) / (double)(n + 1);
            double x = cos(theta);
            double f = (x >= tau) ? 1.0 : low;
            s = s + f * cos((double)k * theta);
        }
        cf[k] = s * ((k == 0 ? 1.0 : 2.0) / (double)(n + 1));
    }
}

void or_cheb_coeffs(int n, double tau, double* cf) { or_cheb_coeffs_lo(n, tau, 0.0, cf); }

/* PS split: argmin d1+d2 with d1 * 2^(d2-1) >= n; ties -> larger d1 */
void or_ps_split(int n, int* d1_out, int* d2_out) {
    int best = 1 << 30, bd1 = 0, bd2 = 0;
    for (int d1 = 1; d1 <= n + 1; d1++) {
        for (int d2 = 1; d2 < 40; d2++) {
            if ((double)d1 * ldexp(1.0, d2 - 1) >= (double)n) {
                if (d1 + d2 < best || (d1 + d2 == best && d1 > bd1)) { best = d1 + d2; bd1 = d1; bd2 = d2; }
                break;
            }
        }
    }
    *d1_out = bd1;
    *d2_out = bd2;
}

/* p (Chebyshev coefficients, length 2M) = q T_M + r, deg q, deg r < M */
static void cheb_split(const double* cf, int len, double* q, double* r) {
    int M = len / 2;
    q[0] = cf[M];
    for (int i = 1; i < M; i++) q[i] = 2.0 * cf[M + i];
    r[0] = cf[0];
    for (int j = 1; j < M; j++) r[j] = cf[j] - cf[2 * M - j];
}

/* FP64 evaluation of the same recursion (used by the pins) */
double or_cheb_ps_eval_fp64(const double* cf, int len, double x) {
    if (len == 2) return cf[0] + cf[1] * x;
    int M = len / 2;
    double* q = (double*)malloc(sizeof(double) * M);
    double* r = (double*)malloc(sizeof(double) * M);
    cheb_split(cf, len, q, r);
    double tm = cos((double)M * acos(x));
    double v = or_cheb_ps_eval_fp64(q, M, x) * tm + or_cheb_ps_eval_fp64(r, M, x);
    free(q);
    free(r);
    return v;
}

typedef struct {
    const or_ctx* c;
    or_keys* k;
    int ls;          /* level of the input score ciphertext */
    u64* x;          /* input ct (T_1) */
    u64** pw;        /* pw[m] = T_{2^m} at level ls - m, m = 1..d2-1 */
} cheb_state;

static size_t ct_words(const or_ctx* c, int l) { return (size_t)2 * (l + 1) * c->n; }

/* returns a freshly allocated ct at level ls - 1 - m, len = 2^(m+1) */
static u64* cheb_eval_rec(cheb_state* S, const double* cf, int len) {
    const or_ctx* c = S->c;
    int ls = S->ls;
    if (len == 2) {
        /* leaf: Rescale(T_1 * round(c1 Delta) + round(c0 Delta) * Delta) */
        double delta = ldexp(1.0, c->scale_bits);
        u64* t = (u64*)malloc(sizeof(u64) * ct_words(c, ls));
        memcpy(t, S->x, sizeof(u64) * ct_words(c, ls));
        mul_int(c, t, ls, llround(cf[1] * delta));
        add_const_res(c, t, ls, llround(cf[0] * delta), 1);
        u64* o = (u64*)malloc(sizeof(u64) * ct_words(c, ls - 1));
        or_rescale(c, t, ls, o);
        free(t);
        return o;
    }
    int M = len / 2, m = 0;
    while ((1 << m) < M) m++;
    double* q = (double*)malloc(sizeof(double) * M);
    double* r = (double*)malloc(sizeof(double) * M);
    cheb_split(cf, len, q, r);
    u64* Q = cheb_eval_rec(S, q, M);   /* level ls - m */
    u64* R = cheb_eval_rec(S, r, M);   /* level ls - m */
    int l = ls - m;
    u64* prod = (u64*)malloc(sizeof(u64) * ct_words(c, l));
    or_mul_relin(c, S->k, Q, S->pw[m], l, prod);
    u64* o = (u64*)malloc(sizeof(u64) * ct_words(c, l - 1));
    or_rescale(c, prod, l, o);
    or_drop(c, R, l, l - 1, R);
    or_add(c, o, R, l - 1, o);
    free(q); free(r); free(Q); free(R); free(prod);
    return o;
}

/* sum_k cf[k] T_k(ct) for the degree-n interpolant of f = 1 above tau, `low` below:
 * ct at level ls -> out at level ls - d2; returns d2, or -1 if the PS split has d1 != 2 */
static int cheb_eval_lo(const or_ctx* c, or_keys* k, const u64* ct, int ls, int n, double tau, double low,
                        u64* out) {
    int d1, d2;
    or_ps_split(n, &d1, &d2);
    if (d1 != 2 || d2 < 1 || ls - d2 < 0) return -1;
    int len = 1 << d2;
    double* cf = (double*)calloc(len, sizeof(double));
    or_cheb_coeffs_lo(n, tau, low, cf);
    cheb_state S;
    S.c = c; S.k = k; S.ls = ls;
    S.x = (u64*)malloc(sizeof(u64) * ct_words(c, ls));
    memcpy(S.x, ct, sizeof(u64) * ct_words(c, ls));
    S.pw = (u64**)calloc(d2 + 1, sizeof(u64*));
    /* giant powers T_{2^m} = 2 T_{2^(m-1)}^2 - 1 */
    u64* prev = S.x;
    for (int m = 1; m < d2; m++) {
        int l = ls - (m - 1);
        u64* sq = (u64*)malloc(sizeof(u64) * ct_words(c, l));
        or_mul_relin(c, k, prev, prev, l, sq);
        u64* t = (u64*)malloc(sizeof(u64) * ct_words(c, l - 1));
        or_rescale(c, sq, l, t);
        or_add(c, t, t, l - 1, t);
        add_const_res(c, t, l - 1, -1, 1);
        S.pw[m] = t;
        prev = t;
        free(sq);
    }
    u64* res = cheb_eval_rec(&S, cf, len);
    memcpy(out, res, sizeof(u64) * ct_words(c, ls - d2));
    free(res);
    for (int m = 1; m < d2; m++) free(S.pw[m]);
    free(S.pw); free(S.x); free(cf);
    return d2;
}

/* the paper's GPU comparator: the interpolant of step(x - tau) (Eq. eq:cheb-sign) */
int or_cheb_eval(const or_ctx* c, or_keys* k, const u64* ct, int ls, int n, double tau, u64* out) {
    return cheb_eval_lo(c, k, ct, ls, n, tau, 0.0, out);
}

/* ------------------------------------------------------------------------ */
/* Hybrid comparator (Section "HyDia": a lower-depth Chebyshev approximation  */
/* followed by a fixed-degree polynomial of Cheon et al. 2020; reading R27):  */
/*   y = the degree-n Chebyshev interpolant of sign(x - tau), as above;       */
/*   out = (1 + f_4(y)) / 2 with f_4(y) = sum_{i=0}^{4} C(2i, i) 4^-i y (1 - y^2)^i */
/*       = (315 y - 420 y^3 + 378 y^5 - 180 y^7 + 35 y^9) / 128,              */
/* the odd polynomial with f_4'(y) = (315/128)(1 - y^2)^4 and f_4(1) = 1, which  */
/* pushes every y near +-1 closer to +-1.                                     */
/* (1 + f_4(y)) / 2 = 1/2 + sum_k a_k y^k, a_k = coefficient / 256, in depth 4:  */
/*   y2 = y y, y4 = y2 y2, y8 = y4 y4 (each rescaled);                          */
/*   u_k = Rescale(y round(a_k Delta)), u_1 with the constant round(Delta/2) Delta; */
/*   t3 = u3 y2, v7 = u7 y2, t5 = u5 y4, t7 = v7 y4, t9 = u9 y8 (each rescaled);  */
/*   out = t9 + t7 + t5 + t3 + u1 at level l - 4 (higher terms dropped to it).   */
/* ------------------------------------------------------------------------ */
static const int F4_NUM[5] = {315, -420, 378, -180, 35};   /* of y, y^3, y^5, y^7, y^9; / 128 */

/* ct * round(v) + round(cst) Delta (in c0), then Rescale: level l -> l - 1 */
static void scalar_rescale(const or_ctx* c, const u64* ct, int l, double v, double cst, u64* out) {
    double delta = ldexp(1.0, c->scale_bits);
    u64* t = (u64*)malloc(sizeof(u64) * ct_words(c, l));
    memcpy(t, ct, sizeof(u64) * ct_words(c, l));
    mul_int(c, t, l, llround(v * delta));
    if (cst != 0.0) add_const_res(c, t, l, llround(cst * delta), 1);
    or_rescale(c, t, l, out);
    free(t);
}

/* a (x) b with relinearisation at level l, then Rescale: -> level l - 1 */
static void mul_rescale(const or_ctx* c, or_keys* k, const u64* a, const u64* b, int l, u64* out) {
    u64* p = (u64*)malloc(sizeof(u64) * ct_words(c, l));
    or_mul_relin(c, k, a, b, l, p);
    or_rescale(c, p, l, out);
    free(p);
}

/* a copy of ct at level l dropped to level l2 <= l */
static u64* dropped(const or_ctx* c, const u64* ct, int l, int l2) {
    u64* o = (u64*)malloc(sizeof(u64) * ct_words(c, l));
    memcpy(o, ct, sizeof(u64) * ct_words(c, l));
    if (l2 < l) or_drop(c, o, l, l2, o);
    return o;
}

/* (1 + f_4(y)) / 2 of y at level l -> out at level l - 4; -1 if l < 4 */
int or_f4_eval(const or_ctx* c, or_keys* k, const u64* y, int l, u64* out) {
    if (l < 4) return -1;
    u64* y2 = (u64*)malloc(sizeof(u64) * ct_words(c, l - 1));
    u64* y4 = (u64*)malloc(sizeof(u64) * ct_words(c, l - 2));
    u64* y8 = (u64*)malloc(sizeof(u64) * ct_words(c, l - 3));
    mul_rescale(c, k, y, y, l, y2);
    mul_rescale(c, k, y2, y2, l - 1, y4);
    mul_rescale(c, k, y4, y4, l - 2, y8);
    u64* u[5];
    for (int i = 0; i < 5; i++) {
        u[i] = (u64*)malloc(sizeof(u64) * ct_words(c, l - 1));
        scalar_rescale(c, y, l, (double)F4_NUM[i] / 256.0, i == 0 ? 0.5 : 0.0, u[i]);
    }
    u64* t3 = (u64*)malloc(sizeof(u64) * ct_words(c, l - 2));
    u64* v7 = (u64*)malloc(sizeof(u64) * ct_words(c, l - 2));
    u64* t5 = (u64*)malloc(sizeof(u64) * ct_words(c, l - 3));
    u64* t7 = (u64*)malloc(sizeof(u64) * ct_words(c, l - 3));
    u64* t9 = (u64*)malloc(sizeof(u64) * ct_words(c, l - 4));
    mul_rescale(c, k, u[1], y2, l - 1, t3);
    mul_rescale(c, k, u[3], y2, l - 1, v7);
    u64* u5 = dropped(c, u[2], l - 1, l - 2);
    mul_rescale(c, k, u5, y4, l - 2, t5);
    mul_rescale(c, k, v7, y4, l - 2, t7);
    u64* u9 = dropped(c, u[4], l - 1, l - 3);
    mul_rescale(c, k, u9, y8, l - 3, t9);
    /* sum at level l - 4 */
    u64* a7 = dropped(c, t7, l - 3, l - 4);
    u64* a5 = dropped(c, t5, l - 3, l - 4);
    u64* a3 = dropped(c, t3, l - 2, l - 4);
    u64* a1 = dropped(c, u[0], l - 1, l - 4);
    or_add(c, t9, a7, l - 4, out);
    or_add(c, out, a5, l - 4, out);
    or_add(c, out, a3, l - 4, out);
    or_add(c, out, a1, l - 4, out);
    for (int i = 0; i < 5; i++) free(u[i]);
    free(y2); free(y4); free(y8); free(t3); free(v7); free(t5); free(t7); free(t9);
    free(u5); free(u9); free(a7); free(a5); free(a3); free(a1);
    return 4;
}

/* Threshold of the match: comparator 0, the paper's GPU path (step interpolant, depth d2);
 * comparator 1, the hybrid (sign interpolant then (1 + f_4) / 2, depth d2 + 4).
 * ct at level ls -> out at level ls - depth; returns the depth or -1. */
int or_comparator_eval(const or_ctx* c, or_keys* k, const u64* ct, int ls, int n, double tau, int comparator,
                       u64* out) {
    if (comparator == 0) return cheb_eval_lo(c, k, ct, ls, n, tau, 0.0, out);
    if (comparator != 1) return -1;
    int d1, d2;
    or_ps_split(n, &d1, &d2);
    if (d1 != 2 || ls - d2 - 4 < 0) return -1;
    u64* y = (u64*)malloc(sizeof(u64) * ct_words(c, ls - d2));
    if (cheb_eval_lo(c, k, ct, ls, n, tau, -1.0, y) < 0) { free(y); return -1; }
    int r = or_f4_eval(c, k, y, ls - d2, out);
    free(y);
    return r < 0 ? -1 : d2 + 4;
}

/* ------------------------------------------------------------------------ */
/* RotateAndSum / EvalSum (Algorithm 5 aggregation; Algorithm 9): for        */
/* t = 0..steps-1: ct <- ct + Rot_{2^t}(ct).                                 */
/* ------------------------------------------------------------------------ */
void or_rotate_sum(const or_ctx* c, const or_keys* k, u64* ct, int l, int steps) {
    u64* r = (u64*)malloc(sizeof(u64) * ct_words(c, l));
    for (int t = 0; t < steps; t++) {
        or_rotate(c, k, ct, l, 1L << t, r);
        or_add(c, ct, r, l, ct);
    }
    free(r);
}

/* RotateAndSum in radix r (a power of two): with s = 1, r, r^2, ... below 2^steps, each step
 * x <- x + sum_{t=1}^{rr-1} Rot_{t s}(x), rr = min(r, 2^steps / s), the rr-1 rotations hoisted
 * over one decomposition of x (Section "Hoisting and double hoisting"). Same total in every
 * slot as the radix-2 form; r = 2 is or_rotate_sum itself. */
int or_rotate_sum_radix(const or_ctx* c, const or_keys* k, u64* ct, int l, int steps, int r) {
    if (r < 2 || (r & (r - 1))) return -1;
    if (r == 2) { or_rotate_sum(c, k, ct, l, steps); return 0; }
    long n = 1L << steps;
    size_t w = ct_words(c, l);
    long* rots = (long*)malloc(sizeof(long) * r);
    u64* rt = (u64*)malloc(sizeof(u64) * w * r);
    for (long s_ = 1; s_ < n; s_ *= r) {
        long rr = n / s_ < r ? n / s_ : r;
        for (long t = 1; t < rr; t++) rots[t - 1] = t * s_;
        or_hoisted_rotate(c, k, ct, l, rots, (int)(rr - 1), rt);
        for (long t = 1; t < rr; t++) or_add(c, ct, rt + (size_t)(t - 1) * w, l, ct);
    }
    free(rots);
    free(rt);
    return 0;
}

/* RotateAndSum in radix r with the rotations of each step summed before one ModDown (double
 * hoisting after Bossuat et al., Section "Hoisting and double hoisting", applied to the
 * aggregation of Algorithm 5): with s = 1, r, r^2, ... below 2^steps and rr = min(r, 2^steps / s),
 *   x <- x + (sum_t sigma_t(x.b) + ModDown(sum_t IP0_t), ModDown(sum_t IP1_t)),  t = 1 .. rr-1,
 * IP0_t, IP1_t the inner products of the one ModUp of x.a under the automorphism sigma_t of
 * Rot_{t s} with its key (Q_l u P, evaluation form). It differs from or_rotate_sum_radix only in
 * the rounding of the ModDowns; with rr = 2 (r = 2) every step is one rotation and one addition,
 * bit for bit the radix-2 form. */
int or_rotate_sum_hoisted(const or_ctx* c, const or_keys* k, u64* ct, int l, int steps, int r) {
    if (r < 2 || (r & (r - 1))) return -1;
    int N = c->n, npos = l + 1 + c->np, beta = beta_at(c, l);
    long n = 1L << steps;
    size_t cw = ct_words(c, l), ew = (size_t)npos * N;
    u64* x = (u64*)malloc(sizeof(u64) * cw);
    u64* ext = (u64*)malloc(sizeof(u64) * (size_t)beta * ew);
    u64* evk = (u64*)malloc(sizeof(u64) * evk_words(c));
    u64* a0 = (u64*)malloc(sizeof(u64) * ew);
    u64* a1 = (u64*)malloc(sizeof(u64) * ew);
    u64* s0 = (u64*)malloc(sizeof(u64) * ew);
    u64* s1 = (u64*)malloc(sizeof(u64) * ew);
    u64* t = (u64*)malloc(sizeof(u64) * N);
    u64* md = (u64*)malloc(sizeof(u64) * cw);
    for (long s_ = 1; s_ < n; s_ *= r) {
        long rr = n / s_ < r ? n / s_ : r;
        memcpy(x, ct, sizeof(u64) * cw);
        modup(c, x + (size_t)(l + 1) * N, l, ext);
        memset(s0, 0, sizeof(u64) * ew);
        memset(s1, 0, sizeof(u64) * ew);
        for (long j = 1; j < rr; j++) {
            u64 g = or_galois(c, j * s_);
            or_make_evk(c, k, 0, g, evk);
            keyswitch_ip(c, ext, l, evk, g, a0, a1);
            for (int pos = 0; pos < npos; pos++) {
                u64 q = c->p[ext_limb(c, l, pos)];
                for (int i = 0; i < N; i++) {
                    s0[(size_t)pos * N + i] = madd(s0[(size_t)pos * N + i], a0[(size_t)pos * N + i], q);
                    s1[(size_t)pos * N + i] = madd(s1[(size_t)pos * N + i], a1[(size_t)pos * N + i], q);
                }
            }
            for (int i = 0; i <= l; i++) {   /* sigma_t(x.b), coefficient form */
                u64 q = c->p[i];
                automorph_coef(c, g, q, x + (size_t)i * N, t);
                for (int m = 0; m < N; m++) ct[(size_t)i * N + m] = madd(ct[(size_t)i * N + m], t[m], q);
            }
        }
        moddown(c, s0, l, md);
        moddown(c, s1, l, md + (size_t)(l + 1) * N);
        or_add(c, ct, md, l, ct);
    }
    free(x); free(ext); free(evk); free(a0); free(a1); free(s0); free(s1); free(t); free(md);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* HyDia packing (Section "Diagonal method for rectangular matrices", Fig. 1) */
/* and the pre-rotated diagonal of Eq. eq:prerotation.                       */
/*   diag_d(M_k)[b ell + r] = T[(k B + b) ell + r][(r + d) mod ell]          */
/*   D'[x] = diag_d(M_k)[(x - shift) mod slots]                               */
/* ------------------------------------------------------------------------ */
void or_diag_slots(const float* T, long K, int ell, int slots, long k, int d, long shift, double* z) {
    long B = slots / ell;
    for (long x = 0; x < slots; x++) {
        long y = ((x - shift) % slots + slots) % slots;
        long b = y / ell, r = y % ell;
        long row = (k * B + b) * ell + r;
        z[x] = (row < K) ? (double)T[(size_t)row * ell + ((r + d) % ell)] : 0.0;
    }
}

/* plaintext diagonal as residues, evaluation form, level l: [l+1][N] */
static void diag_pt_eval(const or_ctx* c, const float* T, long K, int ell, long k, int d, long shift, int l,
                         u64* out) {
    int N = c->n, n = N / 2;
    double* z = (double*)malloc(sizeof(double) * n);
    or_diag_slots(T, K, ell, n, k, d, shift, z);
    or_encode(c, z, l, c->scale_bits, out);
    for (int i = 0; i <= l; i++) ntt_fwd(c, i, out + (size_t)i * N);
    free(z);
}

/* ct (coefficient form) -> evaluation form copy */
static void ct_to_eval(const or_ctx* c, const u64* ct, int l, u64* out) {
    int N = c->n;
    memcpy(out, ct, sizeof(u64) * ct_words(c, l));
    for (int t = 0; t < 2; t++)
        for (int i = 0; i <= l; i++) ntt_fwd(c, i, out + ((size_t)t * (l + 1) + i) * N);
}

/* ------------------------------------------------------------------------ */
/* On-demand BSGS with pre-rotated diagonals (Section "BSGS with pre-rotated  */
/* diagonals on GPU", Eq. eq:prerotation, Algorithms 5 and 6):               */
/*   B_i = Rot_i(q), i < n1 (hoisted, Algorithm 1 step 1)                    */
/*   for k < G, j < n2: P = Rescale(sum_i B_i (.) D'_{k, j n1 + i});         */
/*                      S_k += (j > 0 ? Rot_{j n1}(P) : P)                   */
/* scores: out [G][2][L][N] at level L-1 (L = top level).                    */
/* ------------------------------------------------------------------------ */
/* One giant step j of group g (Algorithm 5, inner loop): babies B_i in evaluation
 * form [n1][2][L+1][N] at level L; P = Rescale(sum_{i < n1, j n1 + i < ell} B_i (.) D'_{g, j n1 + i}),
 * written at level L-1 ([2][L][N], coefficient form). */
int or_giant_step(const or_ctx* c, const u64* babies, int L, int n1, const float* T, long K, int ell, long g, int j,
                  u64* P) {
    int N = c->n;
    size_t cw = ct_words(c, L);
    int cnt = (j * n1 + n1 <= ell) ? n1 : ell - j * n1;
    if (cnt <= 0) return -1;
    u64* pts = (u64*)malloc(sizeof(u64) * (size_t)cnt * (L + 1) * N);
    u64* acc = (u64*)malloc(sizeof(u64) * cw);
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < cnt; i++)
        diag_pt_eval(c, T, K, ell, g, j * n1 + i, (long)j * n1, L, pts + (size_t)i * (L + 1) * N);
#pragma omp parallel for schedule(dynamic)
    for (int li = 0; li <= L; li++) {
        u64 q = c->p[li];
        for (int t = 0; t < 2; t++) {
            u64* a = acc + ((size_t)t * (L + 1) + li) * N;
            memset(a, 0, sizeof(u64) * N);
            for (int i = 0; i < cnt; i++) {
                const u64* b = babies + (size_t)i * cw + ((size_t)t * (L + 1) + li) * N;
                const u64* d = pts + ((size_t)i * (L + 1) + li) * N;
                for (int x = 0; x < N; x++) a[x] = madd(a[x], mmul(b[x], d[x], q), q);
            }
            ntt_inv(c, li, a);
        }
    }
    or_rescale(c, acc, L, P);
    free(pts);
    free(acc);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Baby steps kept in Q_l u P (double hoisting of the baby steps, after       */
/* Bossuat et al.; Section "Hoisting and double hoisting"): the rotations    */
/* B_i = Rot_i(q) are left before their ModDown, in the extended basis,      */
/*   B_i = (P sigma_i(q.b) + IP0_i, IP1_i),  B_0 = (P q.b, P q.a)             */
/* (evaluation form over every limb of Q_l u P; P q is zero on the P limbs), */
/* the plaintext diagonals are encoded over every limb of Q_l u P, and each  */
/* giant step takes one ModDown of its sum, then the rescale:                */
/*   P_j = Rescale(ModDown(sum_i B_i (.) D'_{j n1 + i})).                     */
/* ModDown(P x) = x exactly, so with n1 = 1 this is the plain schedule.       */
/* ------------------------------------------------------------------------ */
/* babies [n1][2][npos][N] of the query qct (coefficient form, level L) */
static void babies_pq(const or_ctx* c, const or_keys* k, const u64* qct, int L, int n1, u64* babies) {
    int N = c->n, npos = L + 1 + c->np, beta = beta_at(c, L);
    size_t bw = (size_t)2 * npos * N;
    u64* ext = (u64*)malloc(sizeof(u64) * (size_t)beta * npos * N);
    modup(c, qct + (size_t)(L + 1) * N, L, ext);
    u64* qe = (u64*)malloc(sizeof(u64) * ct_words(c, L));   /* q in evaluation form */
    memcpy(qe, qct, sizeof(u64) * ct_words(c, L));
    for (int t = 0; t < 2; t++)
        for (int i = 0; i <= L; i++) ntt_fwd(c, i, qe + ((size_t)t * (L + 1) + i) * N);
    u64* evk = (u64*)malloc(sizeof(u64) * evk_words(c));
    u64* tmp = (u64*)malloc(sizeof(u64) * N);
    for (int r = 0; r < n1; r++) {
        u64* B = babies + (size_t)r * bw;
        u64 g = or_galois(c, r);
        if (r == 0 || g == 1) {
            memset(B, 0, sizeof(u64) * bw);
        } else {
            or_make_evk(c, k, 0, g, evk);
            keyswitch_ip(c, ext, L, evk, g, B, B + (size_t)npos * N);
        }
        for (int i = 0; i <= L; i++) {   /* + P sigma_r(q.b) (r = 0: P q.b and P q.a) */
            u64 q = c->p[i], Pm = 1 % q;
            for (int j = 0; j < c->np; j++) Pm = mmul(Pm, c->p[c->nq + j] % q, q);
            const u64* b = qe + (size_t)i * N;
            if (r == 0 || g == 1) {
                const u64* a = qe + (size_t)(L + 1 + i) * N;
                for (int x = 0; x < N; x++) {
                    B[(size_t)i * N + x] = mmul(b[x], Pm, q);
                    B[(size_t)(npos + i) * N + x] = mmul(a[x], Pm, q);
                }
            } else {
                automorph_eval(c, g, b, tmp);
                for (int x = 0; x < N; x++) B[(size_t)i * N + x] = madd(B[(size_t)i * N + x], mmul(tmp[x], Pm, q), q);
            }
        }
    }
    free(ext); free(qe); free(evk); free(tmp);
}

/* plaintext diagonal in evaluation form over every limb of Q_l u P: [npos][N] */
static void diag_pt_eval_pq(const or_ctx* c, const float* T, long K, int ell, long k, int d, long shift, int l,
                            u64* out) {
    int N = c->n, n = N / 2, npos = l + 1 + c->np;
    double* z = (double*)malloc(sizeof(double) * n);
    int64_t* m = (int64_t*)malloc(sizeof(int64_t) * N);
    or_diag_slots(T, K, ell, n, k, d, shift, z);
    or_encode_coeffs(c, z, c->scale_bits, m);
    for (int pos = 0; pos < npos; pos++) {
        int li = ext_limb(c, l, pos);
        u64 q = c->p[li];
        for (int x = 0; x < N; x++) out[(size_t)pos * N + x] = mred_s(m[x], q);
        ntt_fwd(c, li, out + (size_t)pos * N);
    }
    free(z); free(m);
}

/* giant step j of group g from babies in Q_L u P: P = Rescale(ModDown(sum_i B_i (.) D'_{g, j n1 + i})),
 * [2][L][N] coefficient form at level L-1 */
static int giant_step_pq(const or_ctx* c, const u64* babies, int L, int n1, const float* T, long K, int ell, long g,
                         int j, u64* P) {
    int N = c->n, npos = L + 1 + c->np;
    size_t bw = (size_t)2 * npos * N;
    int cnt = (j * n1 + n1 <= ell) ? n1 : ell - j * n1;
    if (cnt <= 0) return -1;
    u64* pts = (u64*)malloc(sizeof(u64) * (size_t)cnt * npos * N);
    u64* acc = (u64*)malloc(sizeof(u64) * bw);
    u64* md = (u64*)malloc(sizeof(u64) * ct_words(c, L));
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < cnt; i++)
        diag_pt_eval_pq(c, T, K, ell, g, j * n1 + i, (long)j * n1, L, pts + (size_t)i * npos * N);
#pragma omp parallel for schedule(dynamic)
    for (int pos = 0; pos < npos; pos++) {
        u64 q = c->p[ext_limb(c, L, pos)];
        for (int t = 0; t < 2; t++) {
            u64* a = acc + ((size_t)t * npos + pos) * N;
            memset(a, 0, sizeof(u64) * N);
            for (int i = 0; i < cnt; i++) {
                const u64* b = babies + (size_t)i * bw + ((size_t)t * npos + pos) * N;
                const u64* d = pts + ((size_t)i * npos + pos) * N;
                for (int x = 0; x < N; x++) a[x] = madd(a[x], mmul(b[x], d[x], q), q);
            }
        }
    }
    moddown(c, acc, L, md);
    moddown(c, acc + (size_t)npos * N, L, md + (size_t)(L + 1) * N);
    or_rescale(c, md, L, P);
    free(pts); free(acc); free(md);
    return 0;
}

/* On-demand BSGS over giant steps j_begin <= j < j_end (all steps: 0..n2); the
 * query ct is at level L (the working level), scores come out at level L-1. */
/* the query's babies: Rot_i(q) in evaluation form [n1][2][L+1][N] (pq = 0), or kept in Q_L u P
 * before their ModDown [n1][2][npos][N] (pq = 1) */
static u64* make_babies(const or_ctx* c, const or_keys* k, const u64* qct, int L, int n1, int pq) {
    size_t cw = ct_words(c, L);
    if (pq) {
        u64* b = (u64*)malloc(sizeof(u64) * (size_t)n1 * 2 * (L + 1 + c->np) * c->n);
        babies_pq(c, k, qct, L, n1, b);
        return b;
    }
    long* rots = (long*)malloc(sizeof(long) * n1);
    for (int i = 0; i < n1; i++) rots[i] = i;
    u64* babies = (u64*)malloc(sizeof(u64) * cw * n1);
    or_hoisted_rotate(c, k, qct, L, rots, n1, babies);
    for (int i = 0; i < n1; i++) ct_to_eval(c, babies + (size_t)i * cw, L, babies + (size_t)i * cw);
    free(rots);
    return babies;
}

static int giant_step_any(const or_ctx* c, const u64* babies, int pq, int L, int n1, const float* T, long K, int ell,
                          long g, int j, u64* P) {
    return pq ? giant_step_pq(c, babies, L, n1, T, K, ell, g, j, P) : or_giant_step(c, babies, L, n1, T, K, ell, g, j, P);
}

static int bsgs_scores_range(const or_ctx* c, const or_keys* k, const u64* qct, int L, const float* T, long K, int ell,
                             int n1, int j_begin, int j_end, int pq, u64* out) {
    int N = c->n, n = N / 2;
    if (ell <= 0 || n % ell != 0 || n1 < 1 || n1 > ell || L < 1) return -1;
    int n2 = (ell + n1 - 1) / n1;
    if (j_begin < 0) j_begin = 0;
    if (j_end > n2) j_end = n2;
    long G = (K + n - 1) / n;
    size_t cw1 = ct_words(c, L - 1);
    u64* babies = make_babies(c, k, qct, L, n1, pq);
    u64* P = (u64*)malloc(sizeof(u64) * cw1);
    u64* R = (u64*)malloc(sizeof(u64) * cw1);
    (void)N;
    for (long g = 0; g < G; g++) {
        u64* S = out + (size_t)g * cw1;
        memset(S, 0, sizeof(u64) * cw1);
        for (int j = j_begin; j < j_end; j++) {
            giant_step_any(c, babies, pq, L, n1, T, K, ell, g, j, P);
            if (j > 0) {
                or_rotate(c, k, P, L - 1, (long)j * n1, R);
                or_add(c, S, R, L - 1, S);
            } else {
                or_add(c, S, P, L - 1, S);
            }
        }
    }
    free(babies); free(P); free(R);
    return (int)G;
}

int or_bsgs_scores_range(const or_ctx* c, const or_keys* k, const u64* qct, int L, const float* T, long K, int ell,
                         int n1, int j_begin, int j_end, u64* out) {
    return bsgs_scores_range(c, k, qct, L, T, K, ell, n1, j_begin, j_end, 0, out);
}

int or_bsgs_scores(const or_ctx* c, const or_keys* k, const u64* qct, int L, const float* T, long K, int ell,
                   int n1, u64* out) {
    return bsgs_scores_range(c, k, qct, L, T, K, ell, n1, 0, ell, 0, out);
}

/* the same with the baby steps kept in Q_L u P (pq = 1) or not (0); hoist: giant steps sharing
 * one ModDown per group */
int or_bsgs_scores_pq(const or_ctx* c, const or_keys* k, const u64* qct, int L, const float* T, long K, int ell,
                      int n1, int pq, int hoist, u64* out);

/* On-demand BSGS whose giant-step key switches of one group share a single ModDown (double
 * hoisting after Bossuat et al., Section "Hoisting and double hoisting"): with P_j the
 * rescaled giant-step products at level l = L-1 and IP0_j, IP1_j the inner products of
 * ModUp(P_j.a) under the automorphism of Rot_{j n1} with its key (in Q_l u P, evaluation form),
 *   S_k = P_0 + (sum_{j>=1} sigma_j(P_j.b) + ModDown(sum_{j>=1} IP0_j), ModDown(sum_{j>=1} IP1_j)).
 * With one giant rotation (n2 = 2) this is P_0 + Rot_{n1}(P_1) itself. */
static int bsgs_scores_hoisted(const or_ctx* c, const or_keys* k, const u64* qct, int L, const float* T, long K,
                               int ell, int n1, int pq, u64* out) {
    int N = c->n, n = N / 2;
    if (ell <= 0 || n % ell != 0 || n1 < 1 || n1 > ell || L < 1) return -1;
    int n2 = (ell + n1 - 1) / n1;
    long G = (K + n - 1) / n;
    int l = L - 1, npos = l + 1 + c->np, beta = beta_at(c, l);
    size_t cw1 = ct_words(c, l), ew = (size_t)npos * N;
    u64* babies = make_babies(c, k, qct, L, n1, pq);
    u64* P = (u64*)malloc(sizeof(u64) * cw1);
    u64* ext = (u64*)malloc(sizeof(u64) * (size_t)beta * ew);
    u64* evk = (u64*)malloc(sizeof(u64) * evk_words(c));
    u64* a0 = (u64*)malloc(sizeof(u64) * ew);
    u64* a1 = (u64*)malloc(sizeof(u64) * ew);
    u64* s0 = (u64*)malloc(sizeof(u64) * ew);
    u64* s1 = (u64*)malloc(sizeof(u64) * ew);
    u64* t = (u64*)malloc(sizeof(u64) * N);
    u64* md = (u64*)malloc(sizeof(u64) * cw1);
    for (long g = 0; g < G; g++) {
        u64* S = out + (size_t)g * cw1;
        giant_step_any(c, babies, pq, L, n1, T, K, ell, g, 0, S);
        memset(s0, 0, sizeof(u64) * ew);
        memset(s1, 0, sizeof(u64) * ew);
        for (int j = 1; j < n2; j++) {
            giant_step_any(c, babies, pq, L, n1, T, K, ell, g, j, P);
            u64 gk = or_galois(c, (long)j * n1);
            modup(c, P + (size_t)(l + 1) * N, l, ext);
            or_make_evk(c, k, 0, gk, evk);
            keyswitch_ip(c, ext, l, evk, gk, a0, a1);
            for (int pos = 0; pos < npos; pos++) {
                u64 q = c->p[ext_limb(c, l, pos)];
                for (int x = 0; x < N; x++) {
                    s0[(size_t)pos * N + x] = madd(s0[(size_t)pos * N + x], a0[(size_t)pos * N + x], q);
                    s1[(size_t)pos * N + x] = madd(s1[(size_t)pos * N + x], a1[(size_t)pos * N + x], q);
                }
            }
            for (int i = 0; i <= l; i++) {   /* sigma_j(P_j.b), coefficient form */
                u64 q = c->p[i];
                automorph_coef(c, gk, q, P + (size_t)i * N, t);
                for (int x = 0; x < N; x++) S[(size_t)i * N + x] = madd(S[(size_t)i * N + x], t[x], q);
            }
        }
        if (n2 > 1) {
            moddown(c, s0, l, md);
            moddown(c, s1, l, md + (size_t)(l + 1) * N);
            or_add(c, S, md, l, S);
        }
    }
    free(babies); free(P); free(ext); free(evk); free(a0); free(a1); free(s0); free(s1); free(t); free(md);
    return (int)G;
}

int or_bsgs_scores_hoisted(const or_ctx* c, const or_keys* k, const u64* qct, int L, const float* T, long K, int ell,
                           int n1, u64* out) {
    return bsgs_scores_hoisted(c, k, qct, L, T, K, ell, n1, 0, out);
}

int or_bsgs_scores_pq(const or_ctx* c, const or_keys* k, const u64* qct, int L, const float* T, long K, int ell,
                      int n1, int pq, int hoist, u64* out) {
    return hoist ? bsgs_scores_hoisted(c, k, qct, L, T, K, ell, n1, pq, out)
                 : bsgs_scores_range(c, k, qct, L, T, K, ell, n1, 0, ell, pq, out);
}

/* Sum over the ell diagonals of a table of rotated queries (Eq. equ:diagbsgsgroupsprecomp):
 * S_g = Rescale(sum_{i < ell} rotQ[i] (.) diag_i(M_g)), plain (not pre-rotated) diagonals.
 * rotQ: [ell][2][L+1][N] evaluation form at level L; out: [G][2][L][N] at level L-1. */
static void scores_from_table(const or_ctx* c, const u64* rq, int L, const float* T, long K, int ell, long G,
                              u64* out) {
    int N = c->n;
    size_t cw = ct_words(c, L), cw1 = ct_words(c, L - 1);
    u64* pt = (u64*)malloc(sizeof(u64) * (size_t)(L + 1) * N);
    u64* acc = (u64*)malloc(sizeof(u64) * cw);
    for (long g = 0; g < G; g++) {
        memset(acc, 0, sizeof(u64) * cw);
        for (int d = 0; d < ell; d++) {
            diag_pt_eval(c, T, K, ell, g, d, 0, L, pt);
#pragma omp parallel for collapse(2)
            for (int t = 0; t < 2; t++)
                for (int li = 0; li <= L; li++) {
                    u64 q = c->p[li];
                    u64* a = acc + ((size_t)t * (L + 1) + li) * N;
                    const u64* b = rq + (size_t)d * cw + ((size_t)t * (L + 1) + li) * N;
                    const u64* p = pt + (size_t)li * N;
                    for (int x = 0; x < N; x++) a[x] = madd(a[x], mmul(b[x], p[x], q), q);
                }
        }
        for (int t = 0; t < 2; t++)
            for (int li = 0; li <= L; li++) ntt_inv(c, li, acc + ((size_t)t * (L + 1) + li) * N);
        or_rescale(c, acc, L, out + (size_t)g * cw1);
    }
    free(pt);
    free(acc);
}

/* Naive diagonal method (Eq. equ:diag), one hoisted rotation per diagonal and a
 * single rescale; used by the pins as the textbook reference. */
int or_diag_scores(const or_ctx* c, const or_keys* k, const u64* qct, const float* T, long K, int ell, u64* out) {
    int N = c->n, L = c->nq - 1, n = N / 2;
    if (ell <= 0 || n % ell != 0 || L < 1) return -1;
    long G = (K + n - 1) / n;
    size_t cw = ct_words(c, L);
    long* rots = (long*)malloc(sizeof(long) * ell);
    for (int i = 0; i < ell; i++) rots[i] = i;
    u64* rq = (u64*)malloc(sizeof(u64) * cw * ell);
    or_hoisted_rotate(c, k, qct, L, rots, ell, rq);
    for (int i = 0; i < ell; i++) ct_to_eval(c, rq + (size_t)i * cw, L, rq + (size_t)i * cw);
    scores_from_table(c, rq, L, T, K, ell, G, out);
    free(rots);
    free(rq);
    return (int)G;
}

/* BSGS-Diagonal with the full table of rotated queries (Section "BSGS with
 * precomputation across groups", Algorithm 1):
 *   step 1: rotQ[b] = Rot_b(q) for b < n1, hoisted over one decomposition of q;
 *   steps 2-3: for every baby b, one decomposition of rotQ[b] shared by its giant
 *              rotations rotQ[j n1 + b] = Rot_{j n1}(rotQ[b]), 1 <= j, j n1 + b < ell;
 *   step 4: per group, S_g = Rescale(sum_{i < ell} rotQ[i] (.) diag_i(M_g)).
 * The query ct is at level L; scores come out at level L-1 ([G][2][L][N]). */
int or_table_scores(const or_ctx* c, const or_keys* k, const u64* qct, int L, const float* T, long K, int ell,
                    int n1, u64* out) {
    int N = c->n, n = N / 2;
    if (ell <= 0 || n % ell != 0 || n1 < 1 || n1 > ell || L < 1) return -1;
    int n2 = (ell + n1 - 1) / n1;
    long G = (K + n - 1) / n;
    size_t cw = ct_words(c, L);
    u64* rq = (u64*)malloc(sizeof(u64) * cw * ell);
    long* rots = (long*)malloc(sizeof(long) * (n1 > n2 ? n1 : n2));
    for (int b = 0; b < n1; b++) rots[b] = b;
    or_hoisted_rotate(c, k, qct, L, rots, n1, rq);  /* rotQ[0 .. n1-1], coefficient form */
    u64* giants = (u64*)malloc(sizeof(u64) * cw * n2);
    for (int b = 0; b < n1; b++) {
        int nj = 0;
        for (int j = 1; j < n2 && j * n1 + b < ell; j++) rots[nj++] = (long)j * n1;
        if (nj == 0) continue;
        or_hoisted_rotate(c, k, rq + (size_t)b * cw, L, rots, nj, giants);
        for (int t = 0; t < nj; t++) memcpy(rq + (size_t)((t + 1) * n1 + b) * cw, giants + (size_t)t * cw,
                                            sizeof(u64) * cw);
    }
    for (int i = 0; i < ell; i++) ct_to_eval(c, rq + (size_t)i * cw, L, rq + (size_t)i * cw);
    scores_from_table(c, rq, L, T, K, ell, G, out);
    free(giants);
    free(rots);
    free(rq);
    return (int)G;
}

/* Threshold and aggregation of the G score cts S [G][2][lq][N] at level lq-1 (Algorithm 5
 * lines for the comparison and the sum, Algorithm 6 for identification): mode 1 writes the
 * G cts p(S_k) at level lq-1-d2; mode 2 writes sum_k p(S_k) after RotateAndSum over all slots. */
/* depth of the threshold: d2 of the PS split (+ 4 for the hybrid comparator), -1 if unsupported */
static int comparator_depth(int cheb_n, int comparator) {
    int d1, d2;
    or_ps_split(cheb_n, &d1, &d2);
    if (d1 != 2 || comparator < 0 || comparator > 1) return -1;
    return d2 + (comparator == 1 ? 4 : 0);
}

static int match_tail(const or_ctx* c, or_keys* k, const u64* S, long G, int lq, int mode, int cheb_n, double tau,
                      int comparator, int sum_radix, int hoist_sum, u64* out, int* out_level) {
    int n = c->n / 2;
    int dep = comparator_depth(cheb_n, comparator);
    if (dep < 0 || lq - 1 - dep < 0) return -1;
    int lo = lq - 1 - dep;
    size_t cwo = ct_words(c, lo);
    if (mode == 1) {
        for (long g = 0; g < G; g++)
            or_comparator_eval(c, k, S + (size_t)g * ct_words(c, lq - 1), lq - 1, cheb_n, tau, comparator,
                               out + g * cwo);
        *out_level = lo;
        return (int)G;
    }
    u64* t = (u64*)malloc(sizeof(u64) * cwo);
    memset(out, 0, sizeof(u64) * cwo);
    for (long g = 0; g < G; g++) {
        or_comparator_eval(c, k, S + (size_t)g * ct_words(c, lq - 1), lq - 1, cheb_n, tau, comparator, t);
        or_add(c, out, t, lo, out);
    }
    int steps = 0;
    while ((1 << steps) < n) steps++;
    int rs = hoist_sum ? or_rotate_sum_hoisted(c, k, out, lo, steps, sum_radix)
                       : or_rotate_sum_radix(c, k, out, lo, steps, sum_radix);
    if (rs < 0) { free(t); return -1; }
    *out_level = lo;
    free(t);
    return 1;
}

/* Full match (Algorithms 5 and 6). The top-level query is first dropped to the
 * working level lq (lq = top: the whole chain). schedule 0: on-demand BSGS with
 * pre-rotated diagonals (hoist: the giant steps of a group share one ModDown; babies_pq: the
 * baby steps stay in Q_l u P, one ModDown per giant step); schedule 1: the
 * rotated-query table of Algorithm 1. mode 0: scores (G cts, level
 * lq-1); mode 1: identification (G cts of p(S_k), level lq-1-d2); mode 2:
 * membership (1 ct: sum_k p(S_k), then RotateAndSum over all slots in radix sum_radix; hoist_sum:
 * the rotations of each step share one ModDown).
 * Returns the number of output cts; *out_level receives their level. */
int or_match(const or_ctx* c, or_keys* k, const u64* qct, int lq, const float* T, long K, int ell, int n1, int mode,
             int cheb_n, double tau, int comparator, int schedule, int sum_radix, int hoist, int babies_pq,
             int hoist_sum, u64* out, int* out_level) {
    int top = c->nq - 1, n = c->n / 2;
    if (lq < 1 || lq > top) return -1;
    long G = (K + n - 1) / n;
    u64* q = (u64*)malloc(sizeof(u64) * ct_words(c, top));
    or_drop(c, qct, top, lq, q);
    if (mode == 0) {
        int r = schedule == 1 ? or_table_scores(c, k, q, lq, T, K, ell, n1, out)
                              : or_bsgs_scores_pq(c, k, q, lq, T, K, ell, n1, babies_pq, hoist, out);
        *out_level = lq - 1;
        free(q);
        return r;
    }
    int dep = comparator_depth(cheb_n, comparator);
    if (dep < 0 || lq - 1 - dep < 0) { free(q); return -1; }
    u64* S = (u64*)malloc(sizeof(u64) * ct_words(c, lq - 1) * G);
    int rs = schedule == 1 ? or_table_scores(c, k, q, lq, T, K, ell, n1, S)
                           : or_bsgs_scores_pq(c, k, q, lq, T, K, ell, n1, babies_pq, hoist, S);
    if (rs < 0) { free(S); free(q); return -1; }
    free(q);
    int r = match_tail(c, k, S, G, lq, mode, cheb_n, tau, comparator, sum_radix, hoist_sum, out, out_level);
    free(S);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Encrypted database: the paper's own setting (Section "BSGS with pre-rotated */
/* diagonals on GPU", with the pre-rotation done by the enroller on the       */
/* plaintext before encryption, Section 5.3.3, and lazy relinearisation,      */
/* Sections 4.1 and 5.2):                                                     */
/*   enrollment: E_{k,d} = Enc(Rot_{-j n1}(diag_d(M_k))), d = j n1 + i         */
/*   online, for group k and giant step j:                                     */
/*     (d0,d1,d2) = sum_i B_i (x) E_{k, j n1 + i}  (tensor products summed)     */
/*     P = Rescale((d0,d1) + KS_{s^2}(d2))         (one relinearisation)        */
/*     S_k += Rot_{j n1}(P)   (P itself for j = 0)                             */
/* ------------------------------------------------------------------------ */
/* Enrollment of a K x ell template matrix: the G*ell diagonal cts, [G][ell][2][level+1][N]
 * coefficient form. Diagonal d of group g is the plaintext diagonal, pre-rotated by the enroller
 * when prerotate != 0 (Eq. eq:prerotation, shift (d / n1) n1; Section 5.3.3) and left plain
 * otherwise (the server pre-rotates, or_prerotate_db), encrypted at the top level with
 * seed + g*ell + d and dropped to `level`. */
void or_encrypt_db(const or_ctx* c, const or_keys* k, const float* T, long K, int ell, int n1, int prerotate,
                   u64 seed, int level, u64* out) {
    int N = c->n, n = N / 2, top = c->nq - 1;
    long G = (K + n - 1) / n;
    double* z = (double*)malloc(sizeof(double) * n);
    u64* full = (u64*)malloc(sizeof(u64) * ct_words(c, top));
    for (long g = 0; g < G; g++)
        for (int d = 0; d < ell; d++) {
            or_diag_slots(T, K, ell, n, g, d, prerotate ? (long)(d / n1) * n1 : 0, z);
            or_encrypt(c, k, z, seed + (u64)(g * ell + d), full);
            or_drop(c, full, top, level, out + (size_t)(g * ell + d) * ct_words(c, level));
        }
    free(z);
    free(full);
}

/* Server-side pre-rotation of encrypted diagonals (Section 5.3, offline phase of the GPU
 * variant with pre-rotated diagonals): the plain diagonal cts E [G][ell][2][el+1][N] are dropped
 * to level L, and diagonal d = j n1 + i with j >= 1 is rotated by -j n1 (a key switch with the
 * key of the negative giant step). out: [G][ell][2][L+1][N] coefficient form. */
void or_prerotate_db(const or_ctx* c, const or_keys* k, const u64* E, int el, long G, int ell, int n1, int L,
                     u64* out) {
    size_t ew = ct_words(c, el), cw = ct_words(c, L);
    u64* t = (u64*)malloc(sizeof(u64) * cw);
    for (long g = 0; g < G; g++)
        for (int d = 0; d < ell; d++) {
            u64* o = out + (size_t)(g * ell + d) * cw;
            int j = d / n1;
            if (j == 0) {
                or_drop(c, E + (size_t)(g * ell + d) * ew, el, L, o);
            } else {
                or_drop(c, E + (size_t)(g * ell + d) * ew, el, L, t);
                or_rotate(c, k, t, L, -(long)j * n1, o);
            }
        }
    free(t);
}

/* One giant step j of group g with encrypted diagonals E ([ell][2][el+1][N] coefficient form,
 * el >= L): babies in evaluation form [n1][2][L+1][N] at level L; P written at level L-1. */
int or_enc_giant_step(const or_ctx* c, or_keys* k, const u64* babies, int L, int n1, const u64* E, int el, int ell,
                      int j, u64* P) {
    int N = c->n;
    size_t cw = ct_words(c, L), ew = ct_words(c, el);
    int cnt = (j * n1 + n1 <= ell) ? n1 : ell - j * n1;
    if (cnt <= 0 || el < L) return -1;
    u64* ev = (u64*)malloc(sizeof(u64) * cw * cnt);
    for (int i = 0; i < cnt; i++) {
        or_drop(c, E + (size_t)(j * n1 + i) * ew, el, L, ev + (size_t)i * cw);
        ct_to_eval(c, ev + (size_t)i * cw, L, ev + (size_t)i * cw);
    }
    /* d = (d0, d1) followed by d2: [3][L+1][N] */
    u64* d = (u64*)malloc(sizeof(u64) * (size_t)3 * (L + 1) * N);
#pragma omp parallel for schedule(dynamic)
    for (int li = 0; li <= L; li++) {
        u64 q = c->p[li];
        u64* o0 = d + (size_t)li * N;
        u64* o1 = d + (size_t)(L + 1 + li) * N;
        u64* o2 = d + (size_t)(2 * (L + 1) + li) * N;
        for (int x = 0; x < N; x++) {
            u64 s0 = 0, s1 = 0, s2 = 0;
            for (int i = 0; i < cnt; i++) {
                const u64* b = babies + (size_t)i * cw;
                const u64* e = ev + (size_t)i * cw;
                u64 b0 = b[(size_t)li * N + x], b1 = b[(size_t)(L + 1 + li) * N + x];
                u64 e0 = e[(size_t)li * N + x], e1 = e[(size_t)(L + 1 + li) * N + x];
                s0 = madd(s0, mmul(b0, e0, q), q);
                s1 = madd(s1, madd(mmul(b0, e1, q), mmul(b1, e0, q), q), q);
                s2 = madd(s2, mmul(b1, e1, q), q);
            }
            o0[x] = s0;
            o1[x] = s1;
            o2[x] = s2;
        }
        ntt_inv(c, li, o0);
        ntt_inv(c, li, o1);
        ntt_inv(c, li, o2);
    }
    relin_add(c, k, d + (size_t)2 * (L + 1) * N, L, d);
    or_rescale(c, d, L, P);
    free(ev);
    free(d);
    return 0;
}

/* S += sum_{j>=1} Rot_{j n1}(P_j) with one ModDown for all j (the double-hoisted giant steps of
 * or_bsgs_scores_hoisted): Ps holds P_1 .. P_{n2-1} at level l, coefficient form. */
static void giant_sum_hoisted(const or_ctx* c, const or_keys* k, u64* S, const u64* Ps, int n2, int n1, int l) {
    int N = c->n, npos = l + 1 + c->np, beta = beta_at(c, l);
    size_t cw1 = ct_words(c, l), ew = (size_t)npos * N;
    u64* ext = (u64*)malloc(sizeof(u64) * (size_t)beta * ew);
    u64* evk = (u64*)malloc(sizeof(u64) * evk_words(c));
    u64* a0 = (u64*)malloc(sizeof(u64) * ew);
    u64* a1 = (u64*)malloc(sizeof(u64) * ew);
    u64* s0 = (u64*)calloc(ew, sizeof(u64));
    u64* s1 = (u64*)calloc(ew, sizeof(u64));
    u64* t = (u64*)malloc(sizeof(u64) * N);
    u64* md = (u64*)malloc(sizeof(u64) * cw1);
    for (int j = 1; j < n2; j++) {
        const u64* P = Ps + (size_t)(j - 1) * cw1;
        u64 gk = or_galois(c, (long)j * n1);
        modup(c, P + (size_t)(l + 1) * N, l, ext);
        or_make_evk(c, k, 0, gk, evk);
        keyswitch_ip(c, ext, l, evk, gk, a0, a1);
        for (int pos = 0; pos < npos; pos++) {
            u64 q = c->p[ext_limb(c, l, pos)];
            for (int x = 0; x < N; x++) {
                s0[(size_t)pos * N + x] = madd(s0[(size_t)pos * N + x], a0[(size_t)pos * N + x], q);
                s1[(size_t)pos * N + x] = madd(s1[(size_t)pos * N + x], a1[(size_t)pos * N + x], q);
            }
        }
        for (int i = 0; i <= l; i++) {
            u64 q = c->p[i];
            automorph_coef(c, gk, q, P + (size_t)i * N, t);
            for (int x = 0; x < N; x++) S[(size_t)i * N + x] = madd(S[(size_t)i * N + x], t[x], q);
        }
    }
    if (n2 > 1) {
        moddown(c, s0, l, md);
        moddown(c, s1, l, md + (size_t)(l + 1) * N);
        or_add(c, S, md, l, S);
    }
    free(ext); free(evk); free(a0); free(a1); free(s0); free(s1); free(t); free(md);
}

/* On-demand BSGS over an encrypted database ([G][ell][2][el+1][N]); the query ct is at level L,
 * scores come out at level L-1 ([G][2][L][N]); hoist: the giant steps of a group share one
 * ModDown. */
int or_enc_bsgs_scores(const or_ctx* c, or_keys* k, const u64* qct, int L, const u64* E, int el, long G, int ell,
                       int n1, int hoist, u64* out) {
    int n = c->n / 2;
    if (ell <= 0 || n % ell != 0 || n1 < 1 || n1 > ell || L < 1 || el < L) return -1;
    int n2 = (ell + n1 - 1) / n1;
    size_t cw = ct_words(c, L), cw1 = ct_words(c, L - 1), ew = ct_words(c, el);
    long* rots = (long*)malloc(sizeof(long) * n1);
    for (int i = 0; i < n1; i++) rots[i] = i;
    u64* babies = (u64*)malloc(sizeof(u64) * cw * n1);
    or_hoisted_rotate(c, k, qct, L, rots, n1, babies);
    for (int i = 0; i < n1; i++) ct_to_eval(c, babies + (size_t)i * cw, L, babies + (size_t)i * cw);
    u64* P = (u64*)malloc(sizeof(u64) * cw1);
    u64* R = (u64*)malloc(sizeof(u64) * cw1);
    u64* Ps = hoist ? (u64*)malloc(sizeof(u64) * cw1 * (n2 > 1 ? n2 - 1 : 1)) : NULL;
    for (long g = 0; g < G; g++) {
        u64* S = out + (size_t)g * cw1;
        memset(S, 0, sizeof(u64) * cw1);
        if (hoist) {
            or_enc_giant_step(c, k, babies, L, n1, E + (size_t)g * ell * ew, el, ell, 0, S);
            for (int j = 1; j < n2; j++)
                or_enc_giant_step(c, k, babies, L, n1, E + (size_t)g * ell * ew, el, ell, j, Ps + (size_t)(j - 1) * cw1);
            giant_sum_hoisted(c, k, S, Ps, n2, n1, L - 1);
            continue;
        }
        for (int j = 0; j < n2; j++) {
            or_enc_giant_step(c, k, babies, L, n1, E + (size_t)g * ell * ew, el, ell, j, P);
            if (j > 0) {
                or_rotate(c, k, P, L - 1, (long)j * n1, R);
                or_add(c, S, R, L - 1, S);
            } else {
                or_add(c, S, P, L - 1, S);
            }
        }
    }
    free(rots); free(babies); free(P); free(R); free(Ps);
    return (int)G;
}

/* Full match against an encrypted database at level el (>= lq); modes as in or_match. */
int or_match_enc(const or_ctx* c, or_keys* k, const u64* qct, int lq, const u64* E, int el, long K, int ell, int n1,
                 int mode, int cheb_n, double tau, int sum_radix, int hoist, int hoist_sum, u64* out,
                 int* out_level) {
    int top = c->nq - 1, n = c->n / 2;
    if (lq < 1 || lq > top || el < lq) return -1;
    long G = (K + n - 1) / n;
    u64* q = (u64*)malloc(sizeof(u64) * ct_words(c, top));
    or_drop(c, qct, top, lq, q);
    if (mode == 0) {
        int r = or_enc_bsgs_scores(c, k, q, lq, E, el, G, ell, n1, hoist, out);
        *out_level = lq - 1;
        free(q);
        return r;
    }
    u64* S = (u64*)malloc(sizeof(u64) * ct_words(c, lq - 1) * G);
    int rs = or_enc_bsgs_scores(c, k, q, lq, E, el, G, ell, n1, hoist, S);
    free(q);
    if (rs < 0) { free(S); return -1; }
    int r = match_tail(c, k, S, G, lq, mode, cheb_n, tau, 0, sum_radix, hoist_sum, out, out_level);
    free(S);
    return r;
}

void or_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
int or_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
