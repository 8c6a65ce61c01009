// Engine: device-resident CKKS state, batched homomorphic operations and the
// encrypted 1:N matcher behind the C ABI declared in include/fr.h.
//
// Data layout in HBM
//   ciphertext batch : [B][2][cap][N] u64, evaluation (NTT) form, limbs 0..level
//                      valid (cap >= level+1, dropping a level keeps the buffer)
//   key-switching key: [ndig][2][nq+np][N] u64, Montgomery form (x * 2^64 mod q)
//   template database: [G][ell][nq][N] u64, pre-rotated diagonals (Eq.
//                      eq:prerotation), evaluation + Montgomery form
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <exception>
#include <set>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "../../include/fr.h"
#include "ckks_kernels.h"
#include "fr_host.h"

using frh::u128;

namespace {

thread_local std::string g_last_error;

struct FrError {
    fr_status s;
    std::string msg;
};

[[noreturn]] void raise(fr_status s, const std::string& m) { throw FrError{s, m}; }

void cuda_check(cudaError_t e, const char* what, int line) {
    if (e != cudaSuccess)
        raise(FR_ERR_CUDA, std::string(what) + " (line " + std::to_string(line) + "): " + cudaGetErrorString(e));
}
#define CU(x) cuda_check((x), #x, __LINE__)

template <class F>
fr_status guard(F f) {
    try {
        f();
        return FR_OK;
    } catch (const FrError& e) {
        g_last_error = e.msg;
        return e.s;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return FR_ERR_INTERNAL;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return FR_ERR_INTERNAL;
    }
}

struct Region {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    double ms = 0;
    uint64_t launches = 0;
    uint64_t bytes = 0;  // algorithmic bytes (minimum DRAM reads + writes) of the timed launches
};

}  // namespace

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
struct Server;

struct fr_ctx {
    frh::Ring R;
    int device = 0;
    cudaStream_t stream = nullptr;       // the context stream (API calls are ordered on it)
    cudaStream_t cur = nullptr;          // stream the internal helpers enqueue on
    cudaStream_t side = nullptr;         // second stream for concurrent branches inside a match
    std::vector<cudaEvent_t> evs;        // fork / join events (no timing)
    bool own_stream = false;
    RingDev rd{};
    DevPrime* d_primes = nullptr;
    u64 *d_tw = nullptr, *d_itw = nullptr;  // (twiddle, Shoup quotient) pairs [primes][N][2]
    unsigned* d_rot = nullptr;
    double *d_zr = nullptr, *d_zi = nullptr;
    uint32_t ell = 0, n1 = 0, schedule = 0, cheb_n = 0;
    double tau = 0.5;
    uint64_t budget = 0;
    int d1 = 0, d2 = 0;
    int comparator = 0;                  // 0: step interpolant; 1: hybrid (sign interpolant, then (1 + f_4) / 2)
    int cmp_depth = 0;                   // levels the threshold consumes: d2 (+ 4 for the hybrid)
    int work_level = 0;                  // level of the query inside fr_match
    std::vector<ModUpTab*> d_modup;      // per level: digits_at(level) tables
    std::vector<int*> d_modup_ntt;       // per level: (offset, prime) of the ext positions to transform
    std::vector<int> modup_ntt_n;
    P2QTab* d_p2q = nullptr;
    std::vector<RescaleTab*> d_rescale;  // per level (index level), level >= 1
    u64 *d_pinv = nullptr, *d_pinv_s = nullptr;
    u64 *d_pmod = nullptr, *d_pmod_s = nullptr;  // [P]_{q_i} and Shoup quotients, Q primes
    u64* d_delta = nullptr;              // Delta mod q_i
    std::map<int, u64*> d_cheb;          // per input level: leaf constants [3][nleaves][level+1]
    std::map<int, u64*> d_f4;            // per input level: hybrid comparator constants [3][5][level+1]
    std::vector<std::pair<double, double>> leaves;  // Chebyshev leaves (c0, c1), BFS order
    std::map<u64, u64*> rotkeys;         // galois element -> key
    u64* relin = nullptr;
    size_t key_words = 0;
    int key_level = 0;                   // keys hold Q limbs 0..key_level (the working level) and P
    int key_limbs = 0;                   // key_level + 1 + np
    size_t resident = 0;
    std::vector<void*> owned;            // persistent device allocations
    long long fail_alloc_after = -1;     // failure injection: the device allocation that fails (-1 none)
    std::vector<void*>* defer_free = nullptr;  // frees held back while a two-stream section unwinds
    bool prof = false;
    std::string prof_only;               // profile only the regions whose name starts with this
    std::map<std::string, Region> regions;
    uint64_t launches = 0;
    int host_threads = 1;
    bool use_graphs = true;              // replay fr_match as a CUDA graph after its first call
    uint32_t db_tier = 0;                // 0 auto, 1 stored diagonals, 2 encoded per query, 3 stored coefficients
    int sum_radix = 2;                   // RotateAndSum radix (2: one rotation per step)
    bool hoist_giants = false;           // giant steps of a group share one ModDown
    bool hoist_babies = false;           // baby steps stay in Q_l u P; one ModDown per giant step
    bool hoist_sum = false;              // the rotations of a RotateAndSum step share one ModDown
    std::map<int, DevPrime*> d_primes_ext;  // per level: the primes of the positions of Q_l u P
    double ntt_tune_us[FR_NTT_BUCKETS * FR_NTT_SHAPES] = {};  // tuner times: bucket x shape (forward + inverse)
    std::set<fr_db*> dbs;                // databases loaded and not yet freed
    std::recursive_mutex mu;             // serialises device work of API calls and the serving loop
    Server* server = nullptr;            // continuous-batching loop (fr_match_submit / fr_match_poll)
};

struct fr_keys {
    frh::KeySet ks;
    int logN = 0, nq = 0, np = 0;
};

struct DevBlock {
    fr_ctx* ctx;
    u64* p;
    DevBlock(fr_ctx* c, u64* ptr) : ctx(c), p(ptr) {}
    ~DevBlock();
};

struct fr_ct {
    const fr_ctx* ctx = nullptr;
    int level = 0;
    int cap = 0;
    double scale = 1.0;
    bool on_dev = false;
    std::vector<u64> host;             // coefficient form [2][level+1][N]
    std::shared_ptr<DevBlock> block;   // device storage (shared by a batch)
    u64* dev = nullptr;                // evaluation form [2][cap][N]
};

struct fr_db {
    fr_ctx* ctx = nullptr;
    long long K = 0;
    int ell = 0;
    long long G = 0;
    int tier = 1;            // 1 (A): pre-rotated diagonals stored in HBM (evaluation form, every limb);
                             // 2 (C): encoded per query from the FP32 templates;
                             // 3 (B): rounded integer coefficients stored, residues + NTT per query;
                             // 4 (E): encrypted pre-rotated diagonals (ciphertexts, evaluation form)
    int schedule = 0;        // 0: on-demand BSGS (diagonals pre-rotated by j n1); 1: rotated-query table (plain diagonals)
    int nl = 0;              // limbs per plaintext diagonal: level + 1, or level + 1 + n_p over Q_l u P (hoist_babies)
    u64* diags = nullptr;    // tier 1: [G][ell][level+1][N]; tier 4: [G][ell][2][level+1][N] (Montgomery form)
    float* templates = nullptr;  // tier 2: [K][ell] FP32
    long long* coeffs = nullptr; // tier 3: [G][ell][N] integer coefficients of the diagonals
    size_t bytes = 0;
};

namespace {

// ---------------------------------------------------------------------------
// device memory (stream-ordered pool)
// ---------------------------------------------------------------------------
u64* dalloc(fr_ctx* c, size_t words) {
    if (words == 0) words = 1;
    if (c->fail_alloc_after >= 0 && c->fail_alloc_after-- == 0)
        raise(FR_ERR_HBM_BUDGET, "injected device allocation failure");
    void* p = nullptr;
    CU(cudaMallocAsync(&p, words * sizeof(u64), c->cur));
    return (u64*)p;
}
void dfree(fr_ctx* c, void* p) {
    if (!p) return;
    if (c->defer_free && std::uncaught_exceptions() > 0) {  // unwinding a two-stream section
        c->defer_free->push_back(p);
        return;
    }
    cudaFreeAsync(p, c->cur);
}
struct Tmp {
    fr_ctx* c;
    u64* p;
    Tmp(fr_ctx* cc, size_t words) : c(cc), p(dalloc(cc, words)) {}
    ~Tmp() { dfree(c, p); }
    Tmp(const Tmp&) = delete;
    Tmp& operator=(const Tmp&) = delete;
};
template <class T>
T* upload_persistent(fr_ctx* c, const T* h, size_t count) {
    void* p = nullptr;
    CU(cudaMalloc(&p, sizeof(T) * (count ? count : 1)));
    CU(cudaMemcpy(p, h, sizeof(T) * count, cudaMemcpyHostToDevice));
    c->owned.push_back(p);
    return (T*)p;
}

// profiling regions: a pair of timing events around the launches of a region. Outside stream
// capture they are recorded on the stream; under capture (the profiled graph replay of a match)
// they become event-record nodes of the graph, so the region is timed inside the replay.
inline void prof_record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}
struct Prof {
    fr_ctx* c;
    Region* r = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    Prof(fr_ctx* cc, const char* name, double bytes = 0) : c(cc) {
        if (!c->prof) return;
        if (!c->prof_only.empty() && std::strncmp(name, c->prof_only.c_str(), c->prof_only.size()) != 0) return;
        r = &c->regions[name];
        r->bytes += (uint64_t)bytes;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        prof_record(a, c->cur);
    }
    ~Prof() {
        if (!r) return;
        prof_record(b, c->cur);
        r->pending.emplace_back(a, b);
        r->launches++;
    }
};

PrimeMap pm_level(int level) {
    PrimeMap m{};
    m.period = level + 1;
    for (int i = 0; i <= level; ++i) m.idx[i] = (unsigned char)i;
    return m;
}
PrimeMap pm_ext(const fr_ctx* c, int level) {
    PrimeMap m{};
    const int npos = level + 1 + c->R.np;
    m.period = npos;
    for (int pos = 0; pos < npos; ++pos) m.idx[pos] = (unsigned char)(pos <= level ? pos : c->R.nq + pos - level - 1);
    return m;
}

void ntt(fr_ctx* c, u64* base, long long outer, int inner, int npolys, const PrimeMap& pm, bool inv) {
    Prof p(c, "ntt", 16.0 * npolys * c->R.N);
    PolyBatch b{base, outer, inner, npolys, pm};
    launch_ntt(c->rd, b, inv, c->cur);
    c->launches += 2;
}
// the same transform out of place: poly p read from src + (p / inner) src_outer + (p % inner) N
// (npolys a multiple of inner), written to its place in base
void ntt_from(fr_ctx* c, const u64* src, long long src_outer, u64* base, long long outer, int inner, int npolys,
              const PrimeMap& pm, bool inv) {
    Prof p(c, "ntt", 16.0 * npolys * c->R.N);
    PolyBatch b{base, outer, inner, npolys, pm};
    b.src = src;
    b.src_outer = src_outer;
    launch_ntt(c->rd, b, inv, c->cur);
    c->launches += 2;
}
// two transforms of the same direction in one launch: n polys of (base, outer, inner, pm), then
// n2 polys of (base2, outer2, inner2, pm2)
void ntt_pair(fr_ctx* c, u64* base, long long outer, int inner, int n, const PrimeMap& pm, u64* base2,
              long long outer2, int inner2, int n2, const PrimeMap& pm2, bool inv) {
    Prof p(c, "ntt", 16.0 * (n + n2) * c->R.N);
    PolyBatch b{base, outer, inner, n + n2, pm};
    b.split = n;
    b.base2 = base2;
    b.outer2 = outer2;
    b.inner2 = inner2;
    b.pm2 = pm2;
    launch_ntt(c->rd, b, inv, c->cur);
    c->launches += 2;
}
// forward NTT of the non-own positions of nj ModUp outputs [nj][beta][npos][N]
void ntt_modup(fr_ctx* c, u64* ext, int nj, int level) {
    const int beta = c->R.digits_at(level), npos = level + 1 + c->R.np;
    const int cnt = c->modup_ntt_n[level];
    Prof p(c, "ntt", 16.0 * nj * cnt * c->R.N);
    PolyBatch b{ext, (long long)beta * npos * c->R.N, 1, nj * cnt, PrimeMap{}, c->d_modup_ntt[level], cnt};
    launch_ntt(c->rd, b, false, c->cur);
    c->launches += 2;
}
// all limbs 0..level of a ciphertext batch [B][2][cap][N]
void ntt_cts(fr_ctx* c, u64* p, int B, int level, int cap, bool inv) {
    ntt(c, p, (long long)cap * c->R.N, level + 1, 2 * B * (level + 1), pm_level(level), inv);
}

long long ctw(const fr_ctx* c, int cap) { return 2ll * cap * c->R.N; }

void copy_d2d(fr_ctx* c, u64* dst, const u64* src, size_t words) {
    Prof p(c, "copy", 16.0 * words);
    CU(cudaMemcpyAsync(dst, src, words * sizeof(u64), cudaMemcpyDeviceToDevice, c->cur));
}
// copy limbs 0..level of B cts from cap_s to cap_d layout
void copy_cts(fr_ctx* c, u64* dst, int cap_d, const u64* src, int cap_s, int B, int level) {
    const size_t N = c->R.N;
    Prof p(c, "copy", 16.0 * 2 * B * (level + 1) * N);
    CU(cudaMemcpy2DAsync(dst, cap_d * N * 8, src, cap_s * N * 8, (level + 1) * N * 8, 2 * (size_t)B,
                         cudaMemcpyDeviceToDevice, c->cur));
}

// ---------------------------------------------------------------------------
// hybrid key switching (ModUp -> automorphism -> inner product -> ModDown)
// ---------------------------------------------------------------------------
struct KSReq {
    const u64* c;      // polynomial to switch, evaluation form, limbs 0..level stride N
    const u64* key;
    u32 galois;
    int mode;          // MDJob mode
    const u64* add;
    int add_cap;
    u64* out;
    int out_cap;
    const u64* add2 = nullptr;  // mode 3
    int sum_dst = -1;           // keyswitch_sums: index of the sum the rotation belongs to
};

// inner product + ModDown of up to FR_MAX_JOBS jobs; job j reads its ModUp output ext[j].
// Jobs arrive sorted by key: consecutive jobs with one key form one group whose key
// words are read once.
void ks_finish(fr_ctx* c, int level, const std::vector<const KSReq*>& reqs, const std::vector<const u64*>& ext) {
    const int N = c->R.N, np = c->R.np, nq = c->R.nq;
    const int npos = level + 1 + np, beta = c->R.digits_at(level);
    const int nj = (int)reqs.size();
    Tmp acc(c, (size_t)nj * 2 * npos * N);
    Tmp conv(c, (size_t)nj * 2 * (level + 1) * N);
    IPJobs ij;
    ij.ngroups = 0;
    int distinct_ext = 0;
    for (int j = 0; j < nj; ++j) {
        ij.j[j].ext = ext[j];
        ij.j[j].key = reqs[j]->key;
        ij.j[j].out = acc.p + (size_t)j * 2 * npos * N;
        ij.j[j].galois = reqs[j]->galois;
        ij.j[j].pad = 0;
        if (j == 0 || reqs[j]->key != reqs[j - 1]->key) {
            ij.gkey[ij.ngroups] = reqs[j]->key;
            ij.gstart[ij.ngroups] = j;
            ij.ngroups++;
        }
        bool seen = false;
        for (int i = 0; i < j && !seen; ++i) seen = ext[i] == ext[j];
        distinct_ext += seen ? 0 : 1;
    }
    ij.gstart[ij.ngroups] = nj;
    {
        const double W = 8.0 * N;
        Prof p(c, "ip", W * npos * (ij.ngroups * 2.0 * beta + distinct_ext * (double)beta + nj * 2.0));
        launch_ip(ij, beta, npos, level, c->key_level + 1, c->key_limbs, c->d_primes, pm_ext(c, level), c->R.logN,
                  c->cur);
        c->launches++;
    }
    PrimeMap pmP{};
    pmP.period = np;
    for (int j = 0; j < np; ++j) pmP.idx[j] = (unsigned char)(nq + j);
    ntt(c, acc.p + (size_t)(level + 1) * N, (long long)npos * N, np, nj * 2 * np, pmP, true);
    {
        Prof p(c, "moddown", 8.0 * N * nj * 2.0 * (np + level + 1));
        launch_p2q(acc.p, 2ll * npos * N, npos, level, conv.p, c->d_p2q, N, nj, c->cur);
        c->launches++;
    }
    MDJobs md;
    for (int j = 0; j < nj; ++j) {
        MDJob& m = md.j[j];
        m.acc = acc.p + (size_t)j * 2 * npos * N;
        m.conv = conv.p + (size_t)j * 2 * (level + 1) * N;
        m.add = reqs[j]->add;
        m.add_cap = reqs[j]->add_cap;
        m.out = reqs[j]->out;
        m.out_cap = reqs[j]->out_cap;
        m.mode = reqs[j]->mode;
        m.galois = reqs[j]->galois;
        m.add2 = reqs[j]->add2;
    }
    // forward NTT of the conversions with the combine as its epilogue
    // the region counts the transform's 16 B per coefficient (its butterflies); the fused
    // epilogue's reads of acc and the addend are not added
    Prof p(c, "ntt", 16.0 * nj * 2 * (level + 1) * N);
    PolyBatch pb{conv.p, (long long)(level + 1) * N, level + 1, nj * 2 * (level + 1), pm_level(level)};
    launch_ntt_moddown(c->rd, pb, md, npos, level, c->d_pinv, c->d_pinv_s, c->cur);
    c->launches += 2;
}

// Hybrid key switching of a list of requests. Requests that switch the same
// input polynomial share one ModUp (hoisting, Algorithm 1 step 1); the others
// get one each. Inputs are processed in groups of up to 16, their jobs sorted by
// key so that each key is read once per inner-product launch.
template <class F>
void modup_chunks(fr_ctx* c, int level, const std::vector<KSReq>& reqs, F finish) {
    const int N = c->R.N;
    const int npos = level + 1 + c->R.np, beta = c->R.digits_at(level);
    const size_t L1N = (size_t)(level + 1) * N;
    std::vector<const u64*> ins;
    std::vector<int> in_of(reqs.size());
    for (size_t j = 0; j < reqs.size(); ++j) {
        int u = -1;
        for (size_t i = 0; i < ins.size(); ++i)
            if (ins[i] == reqs[j].c) { u = (int)i; break; }
        if (u < 0) {
            u = (int)ins.size();
            ins.push_back(reqs[j].c);
        }
        in_of[j] = u;
    }
    const int UCH = 16;
    for (size_t u0 = 0; u0 < ins.size(); u0 += UCH) {
        const int nu = (int)std::min<size_t>(UCH, ins.size() - u0);
        // inputs at one stride (the d2 parts of a batch of products, the ciphertexts of a batch)
        // are read in place: the inverse NTT writes their coefficient form straight into `in`,
        // and the ModUp takes the digits' own positions from the inputs themselves. Others are
        // first gathered into a second half of `in`.
        const long long st = nu > 1 ? (long long)(ins[u0 + 1] - ins[u0]) : (long long)L1N;
        bool strided = st > 0;
        for (int u = 1; u < nu && strided; ++u) strided = ins[u0 + u] == ins[u0] + (long long)u * st;
        Tmp in(c, (size_t)(strided ? 1 : 2) * nu * L1N);  // coefficient form [nu], then gathered inputs
        const u64* in_e = ins[u0];
        long long e_job = st;
        if (!strided) {
            u64* g = in.p + (size_t)nu * L1N;
            for (int u = 0; u < nu; ++u) copy_d2d(c, g + (size_t)u * L1N, ins[u0 + u], L1N);
            in_e = g;
            e_job = (long long)L1N;
        }
        ntt_from(c, in_e, e_job, in.p, (long long)L1N, level + 1, nu * (level + 1), pm_level(level), true);
        Tmp ext(c, (size_t)nu * beta * npos * N);
        {
            Prof p(c, "modup", 8.0 * N * nu * (2.0 * (level + 1) + (double)beta * npos));
            launch_modup(in.p, (long long)L1N, in_e, e_job, ext.p, c->d_modup[level], beta, npos, N, nu, c->cur);
            c->launches++;
        }
        ntt_modup(c, ext.p, nu, level);
        std::vector<int> js;
        for (size_t j = 0; j < reqs.size(); ++j)
            if (in_of[j] >= (int)u0 && in_of[j] < (int)u0 + nu) js.push_back((int)j);
        std::stable_sort(js.begin(), js.end(), [&](int a, int b) { return reqs[a].key < reqs[b].key; });
        const size_t JCH = 32;
        for (size_t j0 = 0; j0 < js.size(); j0 += JCH) {
            std::vector<const KSReq*> rq;
            std::vector<const u64*> ex;
            for (size_t t = j0; t < std::min(js.size(), j0 + JCH); ++t) {
                rq.push_back(&reqs[js[t]]);
                ex.push_back(ext.p + (size_t)(in_of[js[t]] - (int)u0) * beta * npos * N);
            }
            finish(rq, ex);
        }
    }
}

void keyswitch(fr_ctx* c, int level, const std::vector<KSReq>& reqs) {
    if (reqs.empty()) return;
    if (level > c->key_level) raise(FR_ERR_LEVEL, "key switching above the context's working level");
    modup_chunks(c, level, reqs,
                 [&](const std::vector<const KSReq*>& rq, const std::vector<const u64*>& ex) { ks_finish(c, level, rq, ex); });
}

// Sums of rotations that share one ModDown per sum (double hoisting after Bossuat et al.):
// out[o] = base[o] + sum over the requests r with r.sum_dst = o of Rot(r), where a request is
// a rotation (mode 1: r.c the a part, r.add its b part, r.galois, r.key). Every request gets
// its own ModUp (hoisted where inputs repeat); the inner products of a sum and P sigma(b) are
// summed straight into one accumulator in Q_l u P (k_ip_sum), and one ModDown with base[o] as
// its addend ends the sum: base + sum_r sigma_r(b_r) + ModDown(sum_r IP_r).
void keyswitch_sums(fr_ctx* c, int level, const std::vector<KSReq>& reqs, const std::vector<const u64*>& base,
                    int base_cap, const std::vector<u64*>& out, int out_cap) {
    if (level > c->key_level) raise(FR_ERR_LEVEL, "key switching above the context's working level");
    const int N = c->R.N, np = c->R.np, nq = c->R.nq;
    const int npos = level + 1 + np, beta = c->R.digits_at(level);
    const int ndst = (int)out.size();
    const size_t aw = (size_t)2 * npos * N;
    Tmp accs(c, (size_t)ndst * aw);
    {
        Prof p(c, "copy", 8.0 * ndst * aw);
        CU(cudaMemsetAsync(accs.p, 0, (size_t)ndst * aw * 8, c->cur));
    }
    const int pbase = nq;
    (void)pbase;
    modup_chunks(c, level, reqs, [&](const std::vector<const KSReq*>& rq, const std::vector<const u64*>& ex) {
        // the jobs of one sum form one group of the summing inner product
        const int nj = (int)rq.size();
        std::vector<int> ord(nj);
        for (int j = 0; j < nj; ++j) {
            if (rq[j]->sum_dst < 0 || rq[j]->sum_dst >= ndst) raise(FR_ERR_INTERNAL, "sum index out of range");
            ord[j] = j;
        }
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return rq[a]->sum_dst < rq[b]->sum_dst; });
        IPSumJobs ij;
        ij.ngroups = 0;
        std::vector<const u64*> keys, exts;
        for (int t = 0; t < nj; ++t) {
            const KSReq* r = rq[ord[t]];
            ij.j[t] = IPJob{ex[ord[t]], r->key, accs.p + (size_t)r->sum_dst * aw, r->galois, 0, r->add};
            if (t == 0 || r->sum_dst != rq[ord[t - 1]]->sum_dst) ij.gstart[ij.ngroups++] = t;
            if (std::find(keys.begin(), keys.end(), r->key) == keys.end()) keys.push_back(r->key);
            if (std::find(exts.begin(), exts.end(), ex[ord[t]]) == exts.end()) exts.push_back(ex[ord[t]]);
        }
        ij.gstart[ij.ngroups] = nj;
        // key words once per distinct key, ext once per distinct input, c0 gathers on the Q
        // positions, accumulators read and written
        Prof p(c, "ip", 8.0 * N * (npos * (keys.size() * 2.0 * beta + exts.size() * (double)beta + 4.0 * ij.ngroups) +
                                   (double)nj * (level + 1)));
        launch_ip_sum(ij, beta, npos, level, c->key_level + 1, c->key_limbs, c->d_primes, pm_ext(c, level), c->R.logN,
                      c->d_pmod, c->d_pmod_s, c->cur);
        c->launches++;
    });
    // one ModDown per sum: P limbs to coefficients, P -> Q conversion, forward NTT + combine
    PrimeMap pmP{};
    pmP.period = np;
    for (int j = 0; j < np; ++j) pmP.idx[j] = (unsigned char)(nq + j);
    ntt(c, accs.p + (size_t)(level + 1) * N, (long long)npos * N, np, ndst * 2 * np, pmP, true);
    Tmp conv(c, (size_t)ndst * 2 * (level + 1) * N);
    {
        Prof p(c, "moddown", 8.0 * N * ndst * 2.0 * (np + level + 1));
        launch_p2q(accs.p, (long long)aw, npos, level, conv.p, c->d_p2q, N, ndst, c->cur);
        c->launches++;
    }
    for (int o0 = 0; o0 < ndst; o0 += FR_MAX_JOBS) {
        const int no = std::min(FR_MAX_JOBS, ndst - o0);
        MDJobs md;
        for (int o = 0; o < no; ++o) {
            MDJob& m = md.j[o];
            m.acc = accs.p + (size_t)(o0 + o) * aw;
            m.conv = conv.p + (size_t)(o0 + o) * 2 * (level + 1) * N;
            m.add = base[o0 + o];
            m.add_cap = base_cap;
            m.out = out[o0 + o];
            m.out_cap = out_cap;
            m.mode = 2;
            m.galois = 1;
            m.add2 = nullptr;
        }
        Prof p(c, "ntt", 16.0 * no * 2 * (level + 1) * N);
        PolyBatch pb{conv.p + (size_t)o0 * 2 * (level + 1) * N, (long long)(level + 1) * N, level + 1,
                     no * 2 * (level + 1), pm_level(level)};
        launch_ntt_moddown(c->rd, pb, md, npos, level, c->d_pinv, c->d_pinv_s, c->cur);
        c->launches += 2;
    }
}

const u64* rot_key(fr_ctx* c, u64 g) {
    auto it = c->rotkeys.find(g);
    if (it == c->rotkeys.end()) raise(FR_ERR_INVALID_ARG, "rotation key not loaded (galois element " + std::to_string(g) + ")");
    return it->second;
}
const u64* relin_key(fr_ctx* c) {
    if (!c->relin) raise(FR_ERR_INVALID_ARG, "relinearisation key not loaded");
    return c->relin;
}

// rotations: in[j] by ks[j] (or, hoisted, in[0] by every ks[j])
void rotate_cts(fr_ctx* c, int level, const std::vector<const u64*>& in, int in_cap, const std::vector<long>& ks,
                const std::vector<u64*>& out, int out_cap, bool hoisted) {
    std::vector<KSReq> reqs;
    const int N = c->R.N;
    for (size_t j = 0; j < ks.size(); ++j) {
        const u64* src = hoisted ? in[0] : in[j];
        const u64 g = frh::galois_of_rotation(c->R, ks[j]);
        if (g == 1) {
            copy_cts(c, out[j], out_cap, src, in_cap, 1, level);
            continue;
        }
        reqs.push_back(KSReq{src + (size_t)in_cap * N, rot_key(c, g), (u32)g, 1, src, in_cap, out[j], out_cap});
    }
    keyswitch(c, level, reqs);
}

// options of the rescale's fused epilogue (EpiRescale modes)
struct RescaleEpi {
    int mode = 0;
    const u64* add = nullptr;
    int add_cap = 0;
    long long add_bs = 0;
    const u64* cres = nullptr;
};

void rescale(fr_ctx* c, const u64* in, int B, int level, int in_cap, u64* out, int out_cap,
             const RescaleEpi& ep = RescaleEpi()) {
    if (level < 1) raise(FR_ERR_LEVEL, "rescale needs level >= 1");
    const int N = c->R.N, l = level;
    Tmp last(c, (size_t)2 * B * N);
    PrimeMap one{};
    one.period = 1;
    one.idx[0] = (unsigned char)l;
    // the last limb of every component, to coefficients (read in place)
    ntt_from(c, in + (size_t)l * N, (long long)in_cap * N, last.p, N, 1, 2 * B, one, true);
    Tmp lifted(c, (size_t)2 * B * l * N);
    {
        Prof p(c, "rescale", 8.0 * N * 2 * B * (1.0 + l));
        launch_rescale_lift(last.p, lifted.p, c->d_rescale[l], l, N, 2 * B, c->cur);
        c->launches++;
    }
    // forward NTT of the lifted limb with the combine as its epilogue
    Prof p(c, "ntt", 16.0 * 2 * B * l * N);
    PolyBatch pb{lifted.p, (long long)l * N, l, 2 * B * l, pm_level(l - 1)};
    launch_ntt_rescale(c->rd, pb, in, in_cap, out, out_cap, c->d_rescale[l], l, ep.mode, ep.add, ep.add_cap, ep.add_bs,
                       ep.cres, c->cur);
    c->launches += 2;
}

// Rescale(T1 round(c1 Delta) + round(c0 Delta) Delta) for nl leaves of each of B cts T1 at level
// l (x: [B][2][x_cap][N]; constants cc [3][nl][l + 1] as cheb_consts lays them out) -> out
// [B nl][2][out_cap][N] at level l - 1, without the leaves in memory: the inverse NTT of T1's last
// limb, the leaves' lifted last limbs from it, and one forward NTT whose epilogue forms each leaf
// limb from T1 and rescales it. Bit for bit the leaves stored, then rescaled.
void leaves_rescaled(fr_ctx* c, const u64* x, int B, int x_cap, int l, int nl, const u64* cc, u64* out,
                     int out_cap) {
    if (l < 1) raise(FR_ERR_LEVEL, "rescale needs level >= 1");
    const int N = c->R.N, L1 = l + 1;
    const u64 *cb = cc, *cb_s = cc + (size_t)nl * L1, *ca = cc + (size_t)2 * nl * L1;
    PrimeMap one{};
    one.period = 1;
    one.idx[0] = (unsigned char)l;
    Tmp u(c, (size_t)2 * B * N);
    ntt_from(c, x + (size_t)l * N, (long long)x_cap * N, u.p, N, 1, 2 * B, one, true);
    Tmp lifted(c, (size_t)B * nl * 2 * l * N);
    {
        Prof p(c, "rescale", 8.0 * N * B * 2.0 * (1.0 + (double)nl * l));
        launch_leaf_lift(u.p, cb, cb_s, ca, nl, L1, lifted.p, c->d_rescale[l], c->R.primes[l], l, N, B, c->cur);
        c->launches++;
    }
    Prof p(c, "ntt", 16.0 * B * nl * 2 * l * N);
    PolyBatch pb{lifted.p, (long long)l * N, l, B * nl * 2 * l, pm_level(l - 1)};
    launch_ntt_leaf_rescale(c->rd, pb, x, ctw(c, x_cap), x_cap, cb, cb_s, ca, nl, L1, out, out_cap, c->d_rescale[l], l,
                            c->cur);
    c->launches += 2;
}

// ---------------------------------------------------------------------------
// ct x ct with relinearisation (no rescale): out_j = relin(a_j (x) b_j)
// ---------------------------------------------------------------------------
void mul_relin(fr_ctx* c, int level, const std::vector<const u64*>& A, int a_cap, const std::vector<const u64*>& Bv,
               int b_cap, const std::vector<u64*>& out, int out_cap) {
    const int N = c->R.N;
    const size_t J = A.size();
    const size_t dw = (size_t)3 * (level + 1) * N;
    const size_t chunk = 16;
    for (size_t j0 = 0; j0 < J; j0 += chunk) {
        const int nj = (int)std::min(chunk, J - j0);
        Tmp d(c, nj * dw);
        TensorJobs tj;
        for (int j = 0; j < nj; ++j) tj.j[j] = TensorJob{A[j0 + j], Bv[j0 + j], d.p + j * dw, a_cap, b_cap};
        {
            Prof p(c, "tensor", 8.0 * N * nj * 7.0 * (level + 1));
            launch_tensor(tj, nj, level, c->d_primes, N, c->cur);
            c->launches++;
        }
        std::vector<KSReq> reqs;
        for (int j = 0; j < nj; ++j)
            reqs.push_back(KSReq{d.p + j * dw + (size_t)2 * (level + 1) * N, relin_key(c), 1u, 2, d.p + j * dw,
                                 level + 1, out[j0 + j], out_cap});
        keyswitch(c, level, reqs);
    }
}

// One ModDown of nj accumulators acc [nj][2][npos][N] (evaluation form over Q_l u P; their P
// limbs are transformed in place), each plus the addend (d0, d1) of d [nj][3][l+1][N] when d is
// not null, then the rescale by q_l: out_j at level l - 1 (job j at out + j out_bs, cap out_cap),
// then the rescale's epilogue modes. The ModDown's conversion and the rescale's lift share one
// forward NTT; the bits equal ModDown, addition and rescale one after the other.
void moddown_rescale(fr_ctx* c, int l, u64* acc, const u64* d, int nj, u64* out, int out_cap, long long out_bs,
                     const RescaleEpi& ep) {
    const int N = c->R.N, np = c->R.np, nq = c->R.nq;
    const int npos = l + 1 + np;
    const size_t aw = (size_t)2 * npos * N;
    PrimeMap pmP{};
    pmP.period = np;
    for (int j = 0; j < np; ++j) pmP.idx[j] = (unsigned char)(nq + j);
    PrimeMap pmL{};
    pmL.period = 1;
    pmL.idx[0] = (unsigned char)l;
    // the last limb of the result before the rescale, in evaluation form (it reads only limb l of
    // acc and d, not the P limbs)
    Tmp z(c, (size_t)nj * 2 * N);
    {
        Prof p(c, "rescale", 8.0 * N * nj * 2.0 * (d ? 3.0 : 2.0));
        launch_rs_last(acc, d, z.p, c->d_pinv, c->d_pinv_s, npos, l, c->d_primes, N, nj, c->cur);
        c->launches++;
    }
    // the P limbs and that last limb to coefficients, in one launch; the P -> Q conversion
    ntt_pair(c, acc + (size_t)(l + 1) * N, (long long)npos * N, np, nj * 2 * np, pmP, z.p, N, 1, 2 * nj, pmL, true);
    Tmp conv(c, (size_t)nj * 2 * (l + 1) * N);
    {
        Prof p(c, "moddown", 8.0 * N * nj * 2.0 * (np + l + 1));
        launch_p2q(acc, (long long)aw, npos, l, conv.p, c->d_p2q, N, nj, c->cur);
        c->launches++;
    }
    // the lift; one forward NTT with the combine as its epilogue
    Tmp y(c, (size_t)nj * 2 * l * N);
    {
        Prof p(c, "rescale", 8.0 * N * nj * 2.0 * (2.0 + 2.0 * l));
        launch_rs_lift(z.p, conv.p, y.p, c->d_pinv, c->d_pinv_s, c->d_rescale[l], c->d_primes, l, N, nj, c->cur);
        c->launches++;
    }
    Prof p(c, "ntt", 16.0 * nj * 2 * l * N);
    PolyBatch pb{y.p, (long long)l * N, l, nj * 2 * l, pm_level(l - 1)};
    launch_ntt_relin_rescale(c->rd, pb, acc, d, npos, l, c->d_pinv, c->d_pinv_s, c->d_rescale[l], out, out_cap, out_bs,
                             ep.mode, ep.add, ep.add_cap, ep.add_bs, ep.cres, c->cur);
    c->launches += 2;
}

// Products of ciphertext pairs at level l, relinearised and rescaled, with the relinearisation's
// ModDown and the rescale sharing one forward NTT: out_j = Rescale(Relin(A_j (x) B_j)) at level
// l - 1, job j at out + j out_bs (cap out_cap), then the epilogue modes of the rescale. Bit-identical
// to mul_relin followed by rescale (every step is exact modular arithmetic and the NTT is
// linear), with 2(l + 1) fewer limb transforms per product.
void mul_relin_rescale(fr_ctx* c, int l, const std::vector<const u64*>& A, int a_cap, const std::vector<const u64*>& Bv,
                       int b_cap, u64* out, int out_cap, long long out_bs, const RescaleEpi& ep = RescaleEpi()) {
    if (l < 1) raise(FR_ERR_LEVEL, "rescale needs level >= 1");
    if (l > c->key_level) raise(FR_ERR_LEVEL, "key switching above the context's working level");
    const int N = c->R.N, np = c->R.np;
    const int npos = l + 1 + np;
    const size_t J = A.size();
    const size_t dw = (size_t)3 * (l + 1) * N, aw = (size_t)2 * npos * N;
    const size_t chunk = 32;  // products per key-switch batch (two ModUp chunks of 16 inputs)
    for (size_t j0 = 0; j0 < J; j0 += chunk) {
        const int nj = (int)std::min(chunk, J - j0);
        Tmp d(c, nj * dw);
        TensorJobs tj;
        for (int j = 0; j < nj; ++j) tj.j[j] = TensorJob{A[j0 + j], Bv[j0 + j], d.p + j * dw, a_cap, b_cap};
        {
            Prof p(c, "tensor", 8.0 * N * nj * 7.0 * (l + 1));
            launch_tensor(tj, nj, l, c->d_primes, N, c->cur);
            c->launches++;
        }
        // ModUp of every d2 and the inner products with the relinearisation key -> acc [nj][2][npos][N]
        Tmp acc(c, (size_t)nj * aw);
        std::vector<KSReq> reqs;
        for (int j = 0; j < nj; ++j)
            reqs.push_back(KSReq{d.p + j * dw + (size_t)2 * (l + 1) * N, relin_key(c), 1u, 2, d.p + j * dw, l + 1,
                                 nullptr, 0});
        int done = 0;
        modup_chunks(c, l, reqs, [&](const std::vector<const KSReq*>& rq, const std::vector<const u64*>& ex) {
            IPJobs ij;
            ij.ngroups = 1;
            ij.gkey[0] = rq[0]->key;
            ij.gstart[0] = 0;
            ij.gstart[1] = (int)rq.size();
            for (size_t t = 0; t < rq.size(); ++t) {
                const int j = (int)(rq[t]->c - (d.p + 2 * (size_t)(l + 1) * N)) / (int)dw;  // job of this request
                ij.j[t] = IPJob{ex[t], rq[t]->key, acc.p + (size_t)j * aw, 1u, 0};
            }
            Prof p(c, "ip", 8.0 * N * npos * (2.0 * c->R.digits_at(l) + (double)rq.size() * (c->R.digits_at(l) + 2.0)));
            launch_ip(ij, c->R.digits_at(l), npos, l, c->key_level + 1, c->key_limbs, c->d_primes, pm_ext(c, l),
                      c->R.logN, c->cur);
            c->launches++;
            done += (int)rq.size();
        });
        if (done != nj) raise(FR_ERR_INTERNAL, "relinearisation jobs lost");
        RescaleEpi ej = ep;
        if (ej.add) ej.add += (size_t)j0 * ej.add_bs;
        moddown_rescale(c, l, acc.p, d.p, nj, out + (size_t)j0 * out_bs, out_cap, out_bs, ej);
    }
}

void add_cts(fr_ctx* c, const u64* a, int a_cap, long long a_bs, const u64* b, int b_cap, long long b_bs, u64* out,
             int o_cap, long long o_bs, int level, int B) {
    Prof p(c, "misc", 8.0 * c->R.N * B * 6.0 * (level + 1));
    launch_add(a, a_cap, a_bs, b, b_cap, b_bs, out, o_cap, o_bs, level, B, c->d_primes, c->R.N, c->cur);
    c->launches++;
}

// ---------------------------------------------------------------------------
// Chebyshev threshold (Paterson-Stockmeyer, d1 = 2): B cts at level ls -> level ls - d2
// ---------------------------------------------------------------------------
const u64* cheb_consts(fr_ctx* c, int ls) {
    auto it = c->d_cheb.find(ls);
    if (it != c->d_cheb.end()) return it->second;
    const int nl = (int)c->leaves.size(), L1 = ls + 1;
    std::vector<u64> h((size_t)3 * nl * L1);
    const double delta = std::ldexp(1.0, c->R.scale_bits);
    for (int leaf = 0; leaf < nl; ++leaf) {
        const int64_t b = std::llround(c->leaves[leaf].second * delta);
        const int64_t a = std::llround(c->leaves[leaf].first * delta);
        for (int i = 0; i < L1; ++i) {
            const u64 q = c->R.primes[i];
            const u64 bres = frh::resid(b, q);
            h[(size_t)leaf * L1 + i] = bres;
            h[(size_t)nl * L1 + (size_t)leaf * L1 + i] = frh::shoup_quot(bres, q);
            const u64 dm = frh::powm(2, (u64)c->R.scale_bits, q);
            h[(size_t)2 * nl * L1 + (size_t)leaf * L1 + i] = frh::mulm(frh::resid(a, q), dm, q);
        }
    }
    u64* d = upload_persistent(c, h.data(), h.size());
    c->d_cheb[ls] = d;
    return d;
}

// Constants of the hybrid comparator's scaled copies at input level l, laid out for
// leaves_rescaled: [3][5][l+1] (round(a_k Delta) residues, their Shoup quotients, and the
// constant round(Delta / 2) Delta in copy 0), a_k = 315, -420, 378, -180, 35 over 256.
const u64* f4_consts(fr_ctx* c, int l) {
    auto it = c->d_f4.find(l);
    if (it != c->d_f4.end()) return it->second;
    static const int num[5] = {315, -420, 378, -180, 35};
    const int L1 = l + 1;
    std::vector<u64> h((size_t)3 * 5 * L1, 0);
    const double delta = std::ldexp(1.0, c->R.scale_bits);
    for (int k = 0; k < 5; ++k) {
        const int64_t b = std::llround((double)num[k] / 256.0 * delta);
        const int64_t a = k == 0 ? std::llround(0.5 * delta) : 0;
        for (int i = 0; i < L1; ++i) {
            const u64 q = c->R.primes[i];
            const u64 bres = frh::resid(b, q);
            h[(size_t)k * L1 + i] = bres;
            h[(size_t)5 * L1 + (size_t)k * L1 + i] = frh::shoup_quot(bres, q);
            const u64 dm = frh::powm(2, (u64)c->R.scale_bits, q);
            h[(size_t)10 * L1 + (size_t)k * L1 + i] = frh::mulm(frh::resid(a, q), dm, q);
        }
    }
    u64* d = upload_persistent(c, h.data(), h.size());
    c->d_f4[l] = d;
    return d;
}

void chebyshev(fr_ctx* c, const u64* x, int B, int ls, int x_cap, u64* out, int out_cap) {
    const int N = c->R.N, d2 = c->d2;
    if (ls - d2 < 0) raise(FR_ERR_LEVEL, "not enough levels for the Chebyshev evaluation");
    if (d2 + 2 > (int)c->evs.size()) raise(FR_ERR_UNSUPPORTED, "Chebyshev degree too large");
    const int nleaves = (int)c->leaves.size();
    // Two concurrent branches: the giant powers T_{2^m} on the current stream, the
    // leaves and the tree on the side stream; tree level s waits for T_{2^s} only. A match
    // profiled by region class runs both branches on one stream, so that no two timed regions
    // overlap; one that times stages only (filter "stage:") keeps both streams, as unprofiled.
    const bool one_stream = c->prof && c->prof_only.compare(0, 6, "stage:") != 0;
    cudaStream_t main = c->cur, side = one_stream ? c->cur : c->side;
    // Declared first, destroyed last. If an exception unwinds this function, the buffers its
    // locals free are held back (dfree) until both branches have finished, so no kernel still
    // queued on either stream can touch memory the pool has taken back.
    struct JoinOnUnwind {
        fr_ctx* c;
        cudaStream_t main, side;
        std::vector<void*> held;
        std::vector<void*>* prev;
        JoinOnUnwind(fr_ctx* cc, cudaStream_t m, cudaStream_t s) : c(cc), main(m), side(s), prev(cc->defer_free) {
            c->defer_free = &held;
        }
        ~JoinOnUnwind() {
            c->defer_free = prev;
            c->cur = main;
            if (held.empty()) return;
            cudaStreamSynchronize(side);
            cudaStreamSynchronize(main);
            for (void* p : held) cudaFreeAsync(p, main);
            cudaGetLastError();
        }
    } join_on_unwind(c, main, side);
    CU(cudaEventRecord(c->evs[0], main));
    CU(cudaStreamWaitEvent(side, c->evs[0], 0));
    // giant powers T_{2^m}, m = 1..d2-1, T_{2^m} at level ls - m
    std::vector<std::unique_ptr<Tmp>> pw(d2);
    std::vector<int> pw_cap(d2, 0);
    const u64* prev = x;
    int prev_cap = x_cap;
    for (int m = 1; m < d2; ++m) {
        const int lv = ls - (m - 1);
        std::vector<const u64*> A;
        for (int b = 0; b < B; ++b) A.push_back(prev + (size_t)b * ctw(c, prev_cap));
        pw[m].reset(new Tmp(c, (size_t)B * ctw(c, lv)));
        pw_cap[m] = lv;
        RescaleEpi dsub;  // T_2k = 2 T_k^2 - 1: doubling and the constant in the rescale's epilogue
        dsub.mode = 2;
        dsub.cres = c->d_delta;
        mul_relin_rescale(c, lv, A, prev_cap, A, prev_cap, pw[m]->p, lv, ctw(c, lv), dsub);
        CU(cudaEventRecord(c->evs[m], main));
        prev = pw[m]->p;
        prev_cap = lv;
    }
    c->cur = side;
    // leaves: Rescale(T_1 round(c1 Delta) + round(c0 Delta) Delta)
    std::unique_ptr<Tmp> v(new Tmp(c, (size_t)B * nleaves * ctw(c, ls)));
    leaves_rescaled(c, x, B, x_cap, ls, nleaves, cheb_consts(c, ls), v->p, ls);
    int vcap = ls;
    // tree: parents i = child(2i) * T_{2^s} + child(2i+1)
    for (int s = 1; s < d2; ++s) {
        CU(cudaStreamWaitEvent(side, c->evs[s], 0));
        const int P = nleaves >> s;
        const int lc = ls - s;
        std::vector<const u64*> A, Bv;
        for (int b = 0; b < B; ++b)
            for (int i = 0; i < P; ++i) {
                A.push_back(v->p + ((size_t)b * 2 * P + 2 * i) * ctw(c, vcap));
                Bv.push_back(pw[s]->p + (size_t)b * ctw(c, pw_cap[s]));
            }
        std::unique_ptr<Tmp> w(new Tmp(c, (size_t)B * P * ctw(c, lc)));
        RescaleEpi addc;  // + child(2i+1), the odd children, in the rescale's epilogue
        addc.mode = 1;
        addc.add = v->p + ctw(c, vcap);
        addc.add_cap = vcap;
        addc.add_bs = 2 * ctw(c, vcap);
        mul_relin_rescale(c, lc, A, vcap, Bv, pw_cap[s], w->p, lc, ctw(c, lc), addc);
        v = std::move(w);
        vcap = lc;
    }
    copy_cts(c, out, out_cap, v->p, vcap, B, ls - d2);
    // join the side branch back into the main stream
    CU(cudaEventRecord(c->evs[d2], side));
    c->cur = main;
    CU(cudaStreamWaitEvent(main, c->evs[d2], 0));
}

// Second part of the hybrid comparator (Section "HyDia": a Chebyshev approximation followed by
// the fixed polynomial f_4 of Cheon et al. 2020): out = (1 + f_4(y)) / 2 for B cts y at level l
// (y: [B][2][y_cap][N]) -> out [B][2][out_cap][N] at level l - 4. With a_k the coefficients of
// f_4 over 2 (315, -420, 378, -180, 35 over 256 for y, y^3, ..., y^9):
//   y2 = y y, y4 = y2 y2, y8 = y4 y4; u_k = Rescale(y round(a_k Delta)) (u_1 with the constant
//   round(Delta / 2) Delta); t3 = u3 y2, v7 = u7 y2, t5 = u5 y4, t7 = v7 y4, t9 = u9 y8 (every
//   product relinearised and rescaled); out = t9 + t7 + t5 + t3 + u1 at level l - 4.
// Products of one level share one key-switch batch (1, 3, 3 and 1 products per ct), each
// relinearised and rescaled through one shared forward NTT (mul_relin_rescale).
void comparator_f4(fr_ctx* c, const u64* y, int B, int l, int y_cap, u64* out, int out_cap) {
    if (l < 4) raise(FR_ERR_LEVEL, "not enough levels for the hybrid comparator");
    const int cap = l + 1;  // every intermediate is stored with l + 1 limb slots
    const size_t cw = (size_t)ctw(c, cap);
    const u64* cc = f4_consts(c, l);
    const int L1 = l + 1;
    // level l: y2 = y^2, and the five scaled copies u_k
    Tmp Y2(c, (size_t)B * cw);
    {
        std::vector<const u64*> A;
        for (int b = 0; b < B; ++b) A.push_back(y + (size_t)b * ctw(c, y_cap));
        mul_relin_rescale(c, l, A, y_cap, A, y_cap, Y2.p, cap, (long long)cw);
    }
    Tmp U(c, (size_t)B * 5 * cw);  // [B][5]: y, y^3, y^5, y^7, y^9 scalars (u1 with the constant 1/2)
    leaves_rescaled(c, y, B, y_cap, l, 5, cc, U.p, cap);
    auto u = [&](int b, int k) { return U.p + ((size_t)b * 5 + k) * cw; };
    // level l - 1: y4 = y2 y2, t3 = u3 y2, v7 = u7 y2 -> R1 [B][3] at level l - 2
    Tmp R1(c, (size_t)B * 3 * cw);
    {
        std::vector<const u64*> A, Bv;
        for (int b = 0; b < B; ++b) {
            const u64* y2 = Y2.p + (size_t)b * cw;
            const u64* a3[3] = {y2, u(b, 1), u(b, 3)};
            for (int t = 0; t < 3; ++t) {
                A.push_back(a3[t]);
                Bv.push_back(y2);
            }
        }
        mul_relin_rescale(c, l - 1, A, cap, Bv, cap, R1.p, cap, (long long)cw);
    }
    auto r1 = [&](int b, int t) { return R1.p + ((size_t)b * 3 + t) * cw; };  // y4, t3, v7
    // level l - 2: y8 = y4 y4, t5 = u5 y4, t7 = v7 y4 -> R2 [B][3] at level l - 3
    Tmp R2(c, (size_t)B * 3 * cw);
    {
        std::vector<const u64*> A, Bv;
        for (int b = 0; b < B; ++b) {
            const u64* y4 = r1(b, 0);
            const u64* a3[3] = {y4, u(b, 2), r1(b, 2)};
            for (int t = 0; t < 3; ++t) {
                A.push_back(a3[t]);
                Bv.push_back(y4);
            }
        }
        mul_relin_rescale(c, l - 2, A, cap, Bv, cap, R2.p, cap, (long long)cw);
    }
    auto r2 = [&](int b, int t) { return R2.p + ((size_t)b * 3 + t) * cw; };  // y8, t5, t7
    // level l - 3: t9 = u9 y8 -> level l - 4
    Tmp R3(c, (size_t)B * cw);
    {
        std::vector<const u64*> A, Bv;
        for (int b = 0; b < B; ++b) {
            A.push_back(u(b, 4));
            Bv.push_back(r2(b, 0));
        }
        mul_relin_rescale(c, l - 3, A, cap, Bv, cap, R3.p, cap, (long long)cw);
    }
    // out = t9 + t7 + t5 + t3 + u1 on limbs 0..l-4
    const int lo = l - 4;
    const long long so = ctw(c, out_cap);
    add_cts(c, R3.p, cap, (long long)cw, R2.p + 2 * cw, cap, 3ll * (long long)cw, out, out_cap, so, lo, B);
    add_cts(c, out, out_cap, so, R2.p + cw, cap, 3ll * (long long)cw, out, out_cap, so, lo, B);
    add_cts(c, out, out_cap, so, R1.p + cw, cap, 3ll * (long long)cw, out, out_cap, so, lo, B);
    add_cts(c, out, out_cap, so, U.p, cap, 5ll * (long long)cw, out, out_cap, so, lo, B);
}

// Threshold of the match on B score cts x at level ls: the Chebyshev interpolant (comparator 0),
// or the hybrid comparator (1): the sign interpolant, then (1 + f_4) / 2. out at ls - cmp_depth.
void threshold(fr_ctx* c, const u64* x, int B, int ls, int x_cap, u64* out, int out_cap) {
    if (c->comparator == 0) {
        chebyshev(c, x, B, ls, x_cap, out, out_cap);
        return;
    }
    const int l = ls - c->d2;
    Tmp y(c, (size_t)B * ctw(c, l + 1));
    chebyshev(c, x, B, ls, x_cap, y.p, l + 1);
    comparator_f4(c, y.p, B, l, l + 1, out, out_cap);
}

// BSGS schedule of a database with G groups. Auto (2) takes the table of Algorithm 1
// when it needs fewer key switches than the on-demand schedule, ell - n1 < G (n2 - 1)
// (Section "Complexity analysis of our BSGS-Diagonal"), and the table fits in HBM.
int choose_schedule(const fr_ctx* c, long long G) {
    if (c->schedule != 2) return (int)c->schedule;
    const long long ell = c->ell, n1 = c->n1, n2 = (ell + n1 - 1) / n1;
    if (ell - n1 >= G * (n2 - 1)) return 0;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
    const size_t table = (size_t)ell * ctw(c, c->work_level + 1) * 8;
    return table + ((size_t)4 << 30) <= free_b ? 1 : 0;
}

// Pre-rotation block of the stored diagonals: n1 for the on-demand schedule (D' of
// Eq. eq:prerotation), ell (no shift) for the table schedule.
int db_n1_enc(const fr_ctx* c, const fr_db* db) { return db->schedule == 1 ? (int)c->ell : (int)c->n1; }

// The primes of the positions of Q_l u P in order (Q limbs 0..l, then the P limbs), on the
// device; made once per level, outside stream capture (fr_setup, fr_load_db).
const DevPrime* primes_ext(fr_ctx* c, int level) {
    auto it = c->d_primes_ext.find(level);
    if (it != c->d_primes_ext.end()) return it->second;
    const PrimeMap m = pm_ext(c, level);
    DevPrime* d = nullptr;
    CU(cudaMalloc(&d, sizeof(DevPrime) * m.period));
    c->owned.push_back(d);
    for (int pos = 0; pos < m.period; ++pos)
        CU(cudaMemcpy(d + pos, c->d_primes + m.idx[pos], sizeof(DevPrime), cudaMemcpyDeviceToDevice));
    c->d_primes_ext[level] = d;
    return d;
}

// Limbs of a plaintext diagonal at the working level: level + 1, or every limb of Q_l u P when
// the baby steps stay in the extended basis (on-demand schedule).
int diag_limbs(const fr_ctx* c, int schedule) {
    return c->work_level + 1 + (c->hoist_babies && schedule == 0 ? c->R.np : 0);
}

// Encode the diagonals of template group g at the working level into dst [ell][nl][N]
// (evaluation + Montgomery form; nl = level + 1, or the positions of Q_l u P when
// nl > level + 1), diagonal d pre-rotated by (d / n1_enc) n1_enc slots (n1_enc = ell: plain
// diagonals).
void encode_group(fr_ctx* c, const float* dT, long long K, long long g, u64* dst, int n1_enc, int nl) {
    const int N = c->R.N, n = N / 2, L = c->work_level, ell = (int)c->ell;
    const int chunk = 64;
    Tmp z(c, (size_t)chunk * n * 2);
    const bool ext = nl > L + 1;
    const PrimeMap pm = ext ? pm_ext(c, L) : pm_level(L);
    const DevPrime* primes = ext ? primes_ext(c, L) : c->d_primes;
    for (int d0 = 0; d0 < ell; d0 += chunk) {
        const int nd = std::min(chunk, ell - d0);
        u64* o = dst + (size_t)d0 * nl * N;
        {
            Prof p(c, "encode", 8.0 * N * nd * nl);
            launch_encode_diags(dT, K, ell, c->R.logN - 1, g, d0, nd, n1_enc, z.p, o, nl, primes,
                                c->R.scale_bits, c->d_rot, c->d_zr, c->d_zi, c->cur);
            c->launches += 4;
        }
        {
            // forward NTT with the Montgomery conversion in its epilogue
            Prof p(c, "ntt", 16.0 * nd * nl * N);
            PolyBatch pb{o, (long long)nl * N, nl, nd * nl, pm};
            launch_ntt_tomont(c->rd, pb, c->cur);
            c->launches += 2;
        }
    }
}

// RotateAndSum of B ciphertexts [B][2][cap][N] in place: ct <- ct + Rot_{2^t}(ct), t = 0..log2(n)-1
void rotate_sum(fr_ctx* c, u64* ct, int cap, int level, int B = 1) {
    const int n = c->R.N / 2, N = c->R.N;
    const size_t cw = (size_t)ctw(c, cap);
    if (c->hoist_sum) {
        // x <- x + sum_{t=1}^{rr-1} Rot_{t s}(x) with one ModDown per step and ciphertext: the
        // rr-1 rotations share the ModUp of x.a, their inner products and P sigma_t(x.b) are summed
        // in Q_l u P, and the ModDown's combine adds x (in place: each word of x is read and
        // written by the same thread of the last launch)
        const int r = std::max(2, c->sum_radix);
        for (long st = 1; st < n; st *= r) {
            const int rr = (int)std::min<long>(r, n / st);
            std::vector<KSReq> reqs;
            std::vector<const u64*> base;
            std::vector<u64*> outs;
            for (int b = 0; b < B; ++b) {
                u64* x = ct + (size_t)b * cw;
                base.push_back(x);
                outs.push_back(x);
                for (int t = 1; t < rr; ++t) {
                    const u64 g = frh::galois_of_rotation(c->R, (long)t * st);
                    KSReq rq{x + (size_t)cap * N, rot_key(c, g), (u32)g, 1, x, cap, nullptr, 0};
                    rq.sum_dst = b;
                    reqs.push_back(rq);
                }
            }
            keyswitch_sums(c, level, reqs, base, cap, outs, cap);
        }
        return;
    }
    if (c->sum_radix > 2) {
        // radix r: x <- x + sum_{t=1}^{rr-1} Rot_{t s}(x), s = 1, r, r^2, ..., rr = min(r, n / s).
        // The rr-1 rotations of a ciphertext share one ModUp (hoisting); each lands in its slot
        // of a per-ciphertext group [x, Rot_s(x), ..., Rot_{(rr-1)s}(x)] that one sum folds back
        // into x. r = 2 is the loop below.
        const int r = c->sum_radix;
        Tmp grp(c, (size_t)B * r * cw);
        for (long st = 1; st < n; st *= r) {
            const int rr = (int)std::min<long>(r, n / st);
            std::vector<KSReq> reqs;
            for (int b = 0; b < B; ++b) {
                const u64* src = ct + (size_t)b * cw;
                u64* g0 = grp.p + (size_t)b * r * cw;
                copy_d2d(c, g0, src, cw);
                for (int t = 1; t < rr; ++t) {
                    const u64 g = frh::galois_of_rotation(c->R, (long)t * st);
                    reqs.push_back(KSReq{src + (size_t)cap * N, rot_key(c, g), (u32)g, 1, src, cap, g0 + (size_t)t * cw, cap});
                }
            }
            keyswitch(c, level, reqs);
            for (int b = 0; b < B; ++b) {
                Prof p(c, "misc", 8.0 * N * 2.0 * (level + 1) * (rr + 1));
                launch_sum(grp.p + (size_t)b * r * cw, cap, (long long)cw, rr, ct + (size_t)b * cw, cap, level, c->d_primes,
                           N, c->cur);
                c->launches++;
            }
        }
        return;
    }
    // x <- x + Rot_{2^t}(x): the addition is the epilogue of each rotation's ModDown, writing
    // into the other of two buffers
    Tmp r(c, (size_t)B * cw);
    u64* buf[2] = {ct, r.p};
    int cur = 0;
    for (long t = 1; t < n; t <<= 1) {
        const u64 g = frh::galois_of_rotation(c->R, t);
        const u64* key = rot_key(c, g);
        std::vector<KSReq> reqs;
        for (int b = 0; b < B; ++b) {
            const u64* src = buf[cur] + (size_t)b * cw;
            KSReq rq{src + (size_t)cap * N, key, (u32)g, 3, src, cap, buf[1 - cur] + (size_t)b * cw, cap};
            rq.add2 = src;
            reqs.push_back(rq);
        }
        keyswitch(c, level, reqs);
        cur = 1 - cur;
    }
    if (cur) copy_d2d(c, ct, r.p, (size_t)B * cw);
}

// ---------------------------------------------------------------------------
// helpers for handles
// ---------------------------------------------------------------------------
fr_ct* new_dev_ct(fr_ctx* c, std::shared_ptr<DevBlock> blk, u64* p, int level, int cap) {
    fr_ct* ct = new fr_ct();
    ct->ctx = c;
    ct->level = level;
    ct->cap = cap;
    ct->scale = std::ldexp(1.0, c->R.scale_bits);
    ct->on_dev = true;
    ct->block = std::move(blk);
    ct->dev = p;
    return ct;
}
// Storage tier B: the rounded integer coefficients [ell][N] of group g's diagonals (same
// encoding as encode_group up to the rounding).
void encode_group_int(fr_ctx* c, const float* dT, long long K, long long g, long long* dst, int n1_enc) {
    const int N = c->R.N, n = N / 2, ell = (int)c->ell;
    const int chunk = 64;
    Tmp z(c, (size_t)chunk * n * 2);
    for (int d0 = 0; d0 < ell; d0 += chunk) {
        const int nd = std::min(chunk, ell - d0);
        Prof p(c, "encode", 8.0 * N * nd);
        launch_encode_diags_int(dT, K, ell, c->R.logN - 1, g, d0, nd, n1_enc, z.p, dst + (size_t)d0 * N,
                                c->R.scale_bits, c->d_rot, c->d_zr, c->d_zi, c->cur);
        c->launches += 4;
    }
}

// Storage tier B, per query: residues of the stored coefficients at the working level, then
// the forward NTT with the Montgomery conversion: dst [ell][nl][N] as encode_group writes.
void expand_group(fr_ctx* c, const long long* src, u64* dst, int nl) {
    const int N = c->R.N, L = c->work_level, ell = (int)c->ell;
    const int chunk = 64;
    const bool ext = nl > L + 1;
    const PrimeMap pm = ext ? pm_ext(c, L) : pm_level(L);
    const DevPrime* primes = ext ? primes_ext(c, L) : c->d_primes;
    for (int d0 = 0; d0 < ell; d0 += chunk) {
        const int nd = std::min(chunk, ell - d0);
        u64* o = dst + (size_t)d0 * nl * N;
        {
            Prof p(c, "encode", 8.0 * N * nd * (1.0 + nl));
            launch_coef_residues(src + (size_t)d0 * N, nd, o, nl, primes, N, c->cur);
            c->launches++;
        }
        Prof p(c, "ntt", 16.0 * nd * nl * N);
        PolyBatch pb{o, (long long)nl * N, nl, nd * nl, pm};
        launch_ntt_tomont(c->rd, pb, c->cur);
        c->launches += 2;
    }
}

std::shared_ptr<DevBlock> new_block(fr_ctx* c, size_t words) { return std::make_shared<DevBlock>(c, dalloc(c, words)); }

// device copy of a ciphertext (evaluation form) with limbs 0..level (level < 0: all);
// host cts are uploaded (only the kept limbs cross the bus)
void to_device(fr_ctx* c, const fr_ct* ct, u64* dst, int cap, int level = -1) {
    const int N = c->R.N;
    if (level < 0) level = ct->level;
    if (ct->on_dev) {
        copy_cts(c, dst, cap, ct->dev, ct->cap, 1, level);
        return;
    }
    const size_t L1 = ct->level + 1, K1 = level + 1;
    CU(cudaMemcpy2DAsync(dst, (size_t)cap * N * 8, ct->host.data(), L1 * N * 8, K1 * N * 8, 2,
                         cudaMemcpyHostToDevice, c->cur));
    ntt_cts(c, dst, 1, level, cap, false);
}

void export_words(fr_ctx* c, const fr_ct* ct, u64* buf) {
    const int N = c->R.N;
    const size_t L1 = ct->level + 1;
    if (!ct->on_dev) {
        std::memcpy(buf, ct->host.data(), 2 * L1 * N * 8);
        return;
    }
    std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
    Tmp t(c, 2 * L1 * N);
    copy_cts(c, t.p, (int)L1, ct->dev, ct->cap, 1, ct->level);
    ntt_cts(c, t.p, 1, ct->level, (int)L1, true);
    CU(cudaMemcpyAsync(buf, t.p, 2 * L1 * N * 8, cudaMemcpyDeviceToHost, c->cur));
    CU(cudaStreamSynchronize(c->cur));
}

void need_device(const fr_ctx* c) {
    if (!c) raise(FR_ERR_INVALID_ARG, "null context");
    if (c->device < 0) raise(FR_ERR_CUDA, "client-only context (device -1) has no GPU state");
}

void check_ct(const fr_ctx* c, const fr_ct* ct) {
    if (!c) raise(FR_ERR_INVALID_ARG, "null context");
    if (!ct) raise(FR_ERR_INVALID_ARG, "null ciphertext");
    if (ct->ctx && ct->ctx != c) raise(FR_ERR_INVALID_ARG, "ciphertext belongs to another context");
    if (ct->level < 0 || ct->level >= c->R.nq) raise(FR_ERR_LEVEL, "ciphertext level out of range");
}

// q^-1 mod 2^64 for odd q (Newton iteration)
u64 inv_mod_2_64(u64 q) {
    u64 inv = 1;
    for (int i = 0; i < 7; ++i) inv *= 2 - q * inv;
    return inv;
}
// 30-bit halves of a residue below 2^60: low half in bits 0..29, high half in bits 32..61
u64 split30_host(u64 x) { return (x & 0x3fffffffull) | ((x >> 30) << 32); }

void build_tables(fr_ctx* c) {
    const frh::Ring& R = c->R;
    const int N = R.N, T = R.total();
    // primes
    std::vector<DevPrime> dp(T);
    for (int i = 0; i < T; ++i) {
        const u64 q = R.primes[i];
        u64 inv = 1;  // Newton iteration for q^-1 mod 2^64
        for (int k = 0; k < 7; ++k) inv *= 2 - q * inv;
        dp[i].q = q;
        dp[i].qinv = inv;
        const u64 r1 = (u64)(((u128)1 << 64) % q);
        dp[i].r2 = frh::mulm(r1, r1, q);
        dp[i].ninv = R.tabs[i].ninv;
        dp[i].ninv_s = frh::shoup_quot(R.tabs[i].ninv, q);
        dp[i].one_s = frh::shoup_quot(1, q);
    }
    c->d_primes = upload_persistent(c, dp.data(), T);
    // twiddles as (w, Shoup quotient) pairs, one 16-byte load per twiddle: [T][N][2]
    std::vector<u64> tw((size_t)2 * T * N), itw((size_t)2 * T * N);
    for (int i = 0; i < T; ++i)
        for (int k = 0; k < N; ++k) {
            const size_t o = 2 * ((size_t)i * N + k);
            tw[o] = R.tabs[i].tw[k];
            tw[o + 1] = R.tabs[i].tws[k];
            itw[o] = R.tabs[i].itw[k];
            itw[o + 1] = R.tabs[i].itws[k];
        }
    c->d_tw = upload_persistent(c, tw.data(), tw.size());
    c->d_itw = upload_persistent(c, itw.data(), itw.size());
    c->rd = RingDev{R.logN, N, T, c->d_primes, (const ulonglong2*)c->d_tw, (const ulonglong2*)c->d_itw};
    c->d_rot = upload_persistent(c, R.rot_group.data(), R.rot_group.size());
    c->d_zr = upload_persistent(c, R.zr.data(), R.zr.size());
    c->d_zi = upload_persistent(c, R.zi.data(), R.zi.size());
    if (R.ndig > 8) raise(FR_ERR_UNSUPPORTED, "more than 8 key-switching digits");
    // ModUp tables per level
    c->d_modup.assign(R.nq, nullptr);
    c->d_modup_ntt.assign(R.nq, nullptr);
    c->modup_ntt_n.assign(R.nq, 0);
    for (int l = 0; l < R.nq; ++l) {
        const int beta = R.digits_at(l), npos = l + 1 + R.np;
        std::vector<ModUpTab> tabs(beta);
        for (int d = 0; d < beta; ++d) {
            ModUpTab& t = tabs[d];
            std::memset(&t, 0, sizeof(t));
            int lo, hi;
            R.digit_range(l, d, &lo, &hi);
            t.lo = lo;
            t.ns = hi - lo;
            if (t.ns > 8) raise(FR_ERR_UNSUPPORTED, "key-switching digit wider than 8 limbs");
            std::vector<int> src;
            for (int i = lo; i < hi; ++i) src.push_back(i);
            for (int i = 0; i < t.ns; ++i) t.src_q[i] = R.primes[lo + i];
            for (int pos = 0; pos < npos; ++pos) {
                const int pi = pos <= l ? pos : R.nq + pos - l - 1;
                const u64 tp = R.primes[pi];
                t.tq[pos] = tp;
                t.tinv[pos] = inv_mod_2_64(tp);
                t.t_one_s[pos] = (u64)(((unsigned __int128)1 << 64) / tp);
                std::vector<u64> ih, ht;
                frh::bconv_consts(R, src, pi, ih, ht);
                for (int i = 0; i < t.ns; ++i) {
                    t.inv_hat[i] = ih[i];
                    t.inv_hat_s[i] = frh::shoup_quot(ih[i], R.primes[lo + i]);
                    t.hat_m[i][pos] = split30_host((u64)(((unsigned __int128)ht[i] << 64) % tp));
                }
            }
        }
        c->d_modup[l] = upload_persistent(c, tabs.data(), tabs.size());
        std::vector<int> nt;
        for (int d = 0; d < beta; ++d)
            for (int pos = 0; pos < npos; ++pos) {
                if (pos >= tabs[d].lo && pos < tabs[d].lo + tabs[d].ns) continue;
                nt.push_back(d * npos + pos);
                nt.push_back(pos <= l ? pos : R.nq + pos - l - 1);
            }
        c->modup_ntt_n[l] = (int)nt.size() / 2;
        c->d_modup_ntt[l] = upload_persistent(c, nt.data(), nt.size());
    }
    // ModDown: P -> Q
    {
        P2QTab t;
        std::memset(&t, 0, sizeof(t));
        t.np = R.np;
        if (R.np > 8) raise(FR_ERR_UNSUPPORTED, "more than 8 special primes");
        std::vector<int> src;
        for (int j = 0; j < R.np; ++j) src.push_back(R.nq + j);
        for (int j = 0; j < R.np; ++j) t.pq[j] = R.primes[R.nq + j];
        std::vector<u64> pinv(R.nq), pinv_s(R.nq), pmod(R.nq), pmod_s(R.nq);
        for (int i = 0; i < R.nq; ++i) {
            t.qq[i] = R.primes[i];
            std::vector<u64> ih, ht;
            frh::bconv_consts(R, src, i, ih, ht);
            t.qinv[i] = inv_mod_2_64(R.primes[i]);
            t.q_one_s[i] = (u64)(((unsigned __int128)1 << 64) / R.primes[i]);
            for (int j = 0; j < R.np; ++j) {
                t.inv_hat[j] = ih[j];
                t.inv_hat_s[j] = frh::shoup_quot(ih[j], t.pq[j]);
                t.hat_m[j][i] = split30_host((u64)(((unsigned __int128)ht[j] << 64) % R.primes[i]));
            }
            u64 P = 1;
            for (int j = 0; j < R.np; ++j) P = frh::mulm(P, t.pq[j] % R.primes[i], R.primes[i]);
            pinv[i] = frh::invm(P, R.primes[i]);
            pinv_s[i] = frh::shoup_quot(pinv[i], R.primes[i]);
            pmod[i] = P;
            pmod_s[i] = frh::shoup_quot(P, R.primes[i]);
        }
        c->d_p2q = upload_persistent(c, &t, 1);
        c->d_pinv = upload_persistent(c, pinv.data(), pinv.size());
        c->d_pinv_s = upload_persistent(c, pinv_s.data(), pinv_s.size());
        c->d_pmod = upload_persistent(c, pmod.data(), pmod.size());
        c->d_pmod_s = upload_persistent(c, pmod_s.data(), pmod_s.size());
    }
    // rescale tables
    c->d_rescale.assign(R.nq, nullptr);
    for (int l = 1; l < R.nq; ++l) {
        RescaleTab t;
        std::memset(&t, 0, sizeof(t));
        const u64 ql = R.primes[l];
        t.half = (ql - 1) / 2;
        for (int i = 0; i < l; ++i) {
            const u64 q = R.primes[i];
            t.q[i] = q;
            t.one_s[i] = frh::shoup_quot(1, q);
            t.ql_mod[i] = ql % q;
            t.qlinv[i] = frh::invm(ql % q, q);
            t.qlinv_s[i] = frh::shoup_quot(t.qlinv[i], q);
        }
        c->d_rescale[l] = upload_persistent(c, &t, 1);
    }
    std::vector<u64> delta(R.nq);
    for (int i = 0; i < R.nq; ++i) delta[i] = frh::powm(2, (u64)R.scale_bits, R.primes[i]);
    c->d_delta = upload_persistent(c, delta.data(), delta.size());
}

void build_leaves(fr_ctx* c) {
    std::vector<double> cf;
    frh::cheb_coeffs((int)c->cheb_n, c->tau, cf, c->comparator == 1 ? -1.0 : 0.0);
    const size_t len = (size_t)1 << c->d2;
    cf.resize(len, 0.0);
    std::vector<std::vector<double>> level{cf};
    while (level[0].size() > 2) {
        std::vector<std::vector<double>> nxt;
        for (auto& v : level) {
            std::vector<double> q, r;
            frh::cheb_split(v, q, r);
            nxt.push_back(q);
            nxt.push_back(r);
        }
        level.swap(nxt);
    }
    c->leaves.clear();
    for (auto& v : level) c->leaves.emplace_back(v[0], v[1]);
}

}  // namespace

DevBlock::~DevBlock() {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    dfree(ctx, p);
}

namespace {
void drop_graphs(const fr_ctx* c, const fr_db* db);  // CUDA graphs of fr_match (defined below)
void serve_shutdown(fr_ctx* c);                       // serving loop (defined below)
void serve_drain_db(fr_ctx* c, const fr_db* db);
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* fr_last_error(void) { return g_last_error.c_str(); }

fr_status fr_setup(const fr_params* prm, fr_ctx** out) {
    return guard([&] {
        if (!prm || !out) raise(FR_ERR_INVALID_ARG, "null argument");
        if (!prm->q_bits || !prm->p_bits || prm->n_q < 2 || prm->n_p < 1)
            raise(FR_ERR_INVALID_ARG, "need at least 2 Q primes and 1 P prime");
        if (prm->n_q + prm->n_p > FR_MAX_PRIMES) raise(FR_ERR_INVALID_ARG, "too many primes");
        std::unique_ptr<fr_ctx> c(new fr_ctx());
        std::string err;
        std::vector<int> qb(prm->q_bits, prm->q_bits + prm->n_q), pb(prm->p_bits, prm->p_bits + prm->n_p);
        if (!frh::ring_init(c->R, (int)prm->log_n, qb, pb, (int)prm->dnum, (int)prm->scale_bits, err))
            raise(FR_ERR_INVALID_ARG, err);
        const uint32_t n = (uint32_t)c->R.N / 2;
        if (prm->ell == 0 || n % prm->ell != 0) raise(FR_ERR_INVALID_ARG, "ell must divide N/2");
        if (prm->n1 == 0 || prm->n1 > prm->ell) raise(FR_ERR_INVALID_ARG, "need 1 <= n1 <= ell");
        if (prm->schedule > 2) raise(FR_ERR_INVALID_ARG, "schedule must be 0 (on demand), 1 (table) or 2 (auto)");
        c->ell = prm->ell;
        c->n1 = prm->n1;
        c->schedule = prm->schedule;
        c->cheb_n = prm->cheb_degree;
        c->tau = prm->threshold;
        c->budget = prm->hbm_budget_bytes;
        if (c->cheb_n > 0) {
            frh::ps_split((int)c->cheb_n, &c->d1, &c->d2);
            if (c->d1 != 2) raise(FR_ERR_UNSUPPORTED, "Chebyshev degree whose PS split has d1 != 2");
            if (prm->comparator > 1) raise(FR_ERR_INVALID_ARG, "comparator must be 0 or 1");
            c->comparator = (int)prm->comparator;
            c->cmp_depth = c->d2 + (c->comparator == 1 ? 4 : 0);
            build_leaves(c.get());
        }
        c->host_threads = std::max(1u, std::thread::hardware_concurrency());
        if (prm->level_mode > 1) raise(FR_ERR_INVALID_ARG, "level_mode must be 0 or 1");
        if (prm->db_tier > 3) raise(FR_ERR_INVALID_ARG, "db_tier must be 0, 1, 2 or 3");
        c->db_tier = prm->db_tier;
        c->sum_radix = prm->sum_radix ? (int)prm->sum_radix : 2;
        if (prm->hoist_giants > 1) raise(FR_ERR_INVALID_ARG, "hoist_giants must be 0 or 1");
        c->hoist_giants = prm->hoist_giants == 1;
        if (prm->hoist_babies > 1) raise(FR_ERR_INVALID_ARG, "hoist_babies must be 0 or 1");
        c->hoist_babies = prm->hoist_babies == 1;
        if (prm->hoist_sum > 1) raise(FR_ERR_INVALID_ARG, "hoist_sum must be 0 or 1");
        c->hoist_sum = prm->hoist_sum == 1;
        if (c->sum_radix < 2 || c->sum_radix > 64 || (c->sum_radix & (c->sum_radix - 1)))
            raise(FR_ERR_INVALID_ARG, "sum_radix must be 0 or a power of two in [2, 64]");
        c->work_level = c->R.nq - 1;
        if (prm->level_mode == 1) c->work_level = std::min(c->R.nq - 1, 2 + (c->cheb_n ? c->cmp_depth : 0));
        if (prm->device < 0) {
            // client-only context: key generation, encryption and decryption on
            // the host; every device operation fails with FR_ERR_CUDA
            c->device = -1;
            *out = c.release();
            return;
        }
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) raise(FR_ERR_CUDA, "no CUDA device available");
        if (prm->device < 0 || prm->device >= ndev) raise(FR_ERR_INVALID_ARG, "device ordinal out of range");
        c->device = prm->device;
        CU(cudaSetDevice(c->device));
        if (prm->cuda_stream) {
            c->stream = (cudaStream_t)prm->cuda_stream;
        } else {
            CU(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
            c->own_stream = true;
        }
        c->cur = c->stream;
        CU(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        c->evs.resize(16);
        for (auto& e : c->evs) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        cudaMemPool_t pool;
        CU(cudaDeviceGetDefaultMemPool(&pool, c->device));
        uint64_t thr = ~0ull;
        CU(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        build_tables(c.get());
        if (c->hoist_babies) primes_ext(c.get(), c->work_level);  // before any capture uses it
        CU(cudaStreamSynchronize(c->cur));
        // NTT tile shapes per batch-size bucket, timed on this GPU (FR_NTT_TUNE=0: defaults)
        const char* tune = std::getenv("FR_NTT_TUNE");
        if (!(tune && tune[0] == '0')) tune_ntt(c->rd, c->cur, c->ntt_tune_us, 3);
        CU(cudaGetLastError());
        *out = c.release();
    });
}

void fr_free(fr_ctx* c) {
    if (!c) return;
    if (c->device < 0) {
        delete c;
        return;
    }
    cudaSetDevice(c->device);
    serve_shutdown(c);
    cudaStreamSynchronize(c->stream);
    cudaStreamSynchronize(c->side);
    drop_graphs(c, nullptr);
    for (fr_db* db : c->dbs) {  // databases still alive keep their handle, not their memory
        cudaFree(db->diags);
        cudaFree(db->templates);
        cudaFree(db->coeffs);
        db->diags = nullptr;
        db->templates = nullptr;
        db->coeffs = nullptr;
        db->ctx = nullptr;
    }
    for (auto& kv : c->rotkeys) cudaFree(kv.second);
    if (c->relin) cudaFree(c->relin);
    for (void* p : c->owned) cudaFree(p);
    for (auto& r : c->regions)
        for (auto& e : r.second.pending) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    for (auto& e : c->evs) cudaEventDestroy(e);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    // workspaces come from the device's default pool, which keeps what it has reserved while
    // contexts run (its release threshold is unbounded); a context that goes hands the unused
    // part back, with the memory its graphs reserved
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    cudaDeviceGraphMemTrim(c->device);
    cudaGetLastError();
    delete c;
}

fr_status fr_rotation_set(uint32_t ell, uint32_t n1, uint32_t slots, fr_keyset which, int membership, int32_t* out,
                          size_t cap, size_t* n) {
    return guard([&] {
        if (!n) raise(FR_ERR_INVALID_ARG, "null count pointer");
        std::vector<long> v;
        if (!frh::rotation_set(ell, n1, slots, (int)which, membership != 0, v))
            raise(FR_ERR_INVALID_ARG, "bad rotation-set arguments");
        *n = v.size();
        for (size_t i = 0; i < v.size() && i < cap && out; ++i) out[i] = (int32_t)v[i];
    });
}

uint64_t fr_rotation_count(uint32_t ell, uint32_t n1, uint64_t groups, uint32_t schedule) {
    if (ell == 0 || n1 == 0) return 0;
    const uint64_t n2 = (ell + n1 - 1) / n1;
    if (schedule == 1) return ell - 1;
    return (n1 - 1) + groups * (n2 - 1);
}

fr_status fr_required_rotations(const fr_ctx* c, fr_mode mode, int32_t* out, size_t cap, size_t* n) {
    return guard([&] {
        if (!c || !n) raise(FR_ERR_INVALID_ARG, "null argument");
        std::vector<long> v;
        const bool radix = mode == FR_MODE_MEMBERSHIP && c->sum_radix > 2;
        frh::rotation_set(c->ell, c->n1, (uint32_t)c->R.N / 2, frh::RV_ONDEMAND, mode == FR_MODE_MEMBERSHIP && !radix, v);
        if (radix) {  // RotateAndSum in radix r: t s for t < r, s = 1, r, r^2, ...
            std::set<long> all(v.begin(), v.end());
            const long ns = c->R.N / 2;
            for (long st = 1; st < ns; st *= c->sum_radix)
                for (long t = 1; t < std::min<long>(c->sum_radix, ns / st); ++t) all.insert(t * st);
            v.assign(all.begin(), all.end());
        }
        *n = v.size();
        for (size_t i = 0; i < v.size() && i < cap && out; ++i) out[i] = (int32_t)v[i];
    });
}

fr_status fr_keygen(fr_ctx* c, const int32_t* rotations, size_t n_rot, uint64_t seed, fr_keys** out) {
    return guard([&] {
        if (!c || !out || (n_rot && !rotations)) raise(FR_ERR_INVALID_ARG, "null argument");
        std::unique_ptr<fr_keys> k(new fr_keys());
        std::vector<u64> gal;
        for (size_t i = 0; i < n_rot; ++i) gal.push_back(frh::galois_of_rotation(c->R, rotations[i]));
        frh::keygen(c->R, seed, gal, k->ks, c->host_threads);
        k->logN = c->R.logN;
        k->nq = c->R.nq;
        k->np = c->R.np;
        *out = k.release();
    });
}

void fr_free_keys(fr_keys* k) { delete k; }

fr_status fr_load_keys(fr_ctx* c, const fr_keys* k) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        if (!c || !k) raise(FR_ERR_INVALID_ARG, "null argument");
        if (k->logN != c->R.logN || k->nq != c->R.nq || k->np != c->R.np)
            raise(FR_ERR_INVALID_ARG, "keys were generated for other parameters");
        CU(cudaSetDevice(c->device));
        // keys are kept only for the limbs the context can switch: Q limbs 0..work level and P
        const int T = c->R.total(), N = c->R.N, nq = c->R.nq, np = c->R.np;
        const int wl = c->work_level, kd = c->R.digits_at(wl), Tk = wl + 1 + np;
        const size_t words = (size_t)kd * 2 * Tk * N;
        c->key_words = words;
        c->key_level = wl;
        c->key_limbs = Tk;
        size_t need = words * 8 * (1 + k->ks.rot.size());
        if (c->budget && c->resident + need > c->budget)
            raise(FR_ERR_HBM_BUDGET, "evaluation keys exceed the HBM budget");
        PrimeMap pm{};
        pm.period = Tk;
        for (int pos = 0; pos < Tk; ++pos) pm.idx[pos] = (unsigned char)(pos <= wl ? pos : nq + pos - wl - 1);
        std::vector<u64> stage(words);
        auto up = [&](const std::vector<u64>& h) {
            for (int d = 0; d < kd; ++d)
                for (int t = 0; t < 2; ++t)
                    for (int pos = 0; pos < Tk; ++pos) {
                        const int src = pos <= wl ? pos : nq + pos - wl - 1;
                        std::memcpy(&stage[(((size_t)d * 2 + t) * Tk + pos) * N], &h[(((size_t)d * 2 + t) * T + src) * N],
                                    (size_t)N * 8);
                    }
            u64* dptr = nullptr;
            CU(cudaMalloc(&dptr, words * 8));
            CU(cudaMemcpy(dptr, stage.data(), words * 8, cudaMemcpyHostToDevice));
            launch_to_mont(dptr, N, pm, c->d_primes, (long long)words, c->cur);
            CU(cudaStreamSynchronize(c->cur));
            return dptr;
        };
        if (!c->relin) {
            c->relin = up(k->ks.relin);
            c->resident += words * 8;
        }
        for (auto& kv : k->ks.rot) {
            if (c->rotkeys.count(kv.first)) continue;
            c->rotkeys[kv.first] = up(kv.second);
            c->resident += words * 8;
        }
    });
}

fr_status fr_load_db(fr_ctx* c, const float* templates, size_t K, size_t ell, fr_db** out) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        if (!c || !templates || !out || K == 0) raise(FR_ERR_INVALID_ARG, "null argument or empty database");
        if (ell != c->ell) raise(FR_ERR_INVALID_ARG, "template dimension differs from the context's ell");
        CU(cudaSetDevice(c->device));
        const int N = c->R.N, n = N / 2;
        std::unique_ptr<fr_db> db(new fr_db());
        db->ctx = c;
        db->K = (long long)K;
        db->ell = (int)ell;
        db->G = ((long long)K + n - 1) / n;
        db->schedule = choose_schedule(c, db->G);
        const int nl = diag_limbs(c, db->schedule);
        db->nl = nl;
        const size_t tbytes = K * ell * sizeof(float);
        const size_t dbytes = (size_t)db->G * ell * nl * N * 8;
        // storage tier: the stored diagonals when they fit (budget, or free HBM minus a working
        // margin of 2 groups of diagonals), else the stored integer coefficients, else the
        // templates and a per-query encode
        const size_t ibytes = (size_t)db->G * ell * N * 8;
        int tier = (int)c->db_tier;
        if (tier == 0) {
            size_t free_b = 0, total_b = 0;
            CU(cudaMemGetInfo(&free_b, &total_b));
            const size_t margin = (size_t)2 * ell * nl * N * 8 + ((size_t)4 << 30);
            auto fits = [&](size_t b) { return c->budget ? c->resident + b <= c->budget : b + margin <= free_b; };
            tier = fits(dbytes) ? 1 : fits(ibytes) ? 3 : 2;
        }
        db->tier = tier;
        db->bytes = tier == 1 ? dbytes : tier == 3 ? ibytes : tbytes;
        if (c->budget && c->resident + db->bytes > c->budget)
            raise(FR_ERR_HBM_BUDGET, "database exceeds the HBM budget");
        float* dT = nullptr;
        CU(cudaMalloc(&dT, tbytes));
        CU(cudaMemcpyAsync(dT, templates, tbytes, cudaMemcpyHostToDevice, c->cur));
        if (tier == 1 || tier == 3) {
            void* p = nullptr;
            cudaError_t e = cudaMalloc(&p, tier == 1 ? dbytes : ibytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                cudaFree(dT);
                raise(e == cudaErrorMemoryAllocation ? FR_ERR_HBM_BUDGET : FR_ERR_CUDA,
                      std::string("cannot hold the database diagonals: ") + cudaGetErrorString(e));
            }
            for (long long g = 0; g < db->G; ++g) {
                if (tier == 1) {
                    db->diags = (u64*)p;
                    encode_group(c, dT, (long long)K, g, db->diags + (size_t)g * ell * nl * N, db_n1_enc(c, db.get()),
                                 nl);
                } else {
                    db->coeffs = (long long*)p;
                    encode_group_int(c, dT, (long long)K, g, db->coeffs + (size_t)g * ell * N, db_n1_enc(c, db.get()));
                }
            }
            CU(cudaStreamSynchronize(c->cur));
            CU(cudaFree(dT));
        } else {
            db->templates = dT;
            CU(cudaStreamSynchronize(c->cur));
        }
        c->resident += db->bytes;
        c->dbs.insert(db.get());
        *out = db.release();
    });
}

fr_status fr_encrypt_db(const fr_ctx* c, const fr_keys* k, const float* templates, size_t K, size_t ell,
                        int prerotate, uint32_t level, uint64_t seed, uint64_t* out, size_t words) {
    return guard([&] {
        if (!c || !k || !templates || !out || K == 0) raise(FR_ERR_INVALID_ARG, "null argument or empty database");
        if (ell != c->ell) raise(FR_ERR_INVALID_ARG, "template dimension differs from the context's ell");
        if ((int)level >= c->R.nq) raise(FR_ERR_LEVEL, "level out of range");
        const size_t N = c->R.N, n = N / 2, G = (K + n - 1) / n;
        if (words < G * ell * 2 * (level + 1) * N) raise(FR_ERR_INVALID_ARG, "output buffer too small");
        const int threads = std::max(1, (int)std::thread::hardware_concurrency());
        frh::encrypt_diagonals(c->R, k->ks, templates, (long long)K, (int)ell, (int)c->n1, prerotate != 0, (int)level,
                               seed, threads, out);
    });
}

fr_status fr_load_db_encrypted(fr_ctx* c, const uint64_t* cts, size_t K, size_t ell, uint32_t level, int prerotated,
                               fr_db** out) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        if (!cts || !out || K == 0) raise(FR_ERR_INVALID_ARG, "null argument or empty database");
        if (ell != c->ell) raise(FR_ERR_INVALID_ARG, "template dimension differs from the context's ell");
        const int L = c->work_level, L1 = L + 1, N = c->R.N, n = N / 2;
        if ((int)level < L || (int)level >= c->R.nq)
            raise(FR_ERR_LEVEL, "diagonal ciphertexts must be at or above the working level");
        CU(cudaSetDevice(c->device));
        std::unique_ptr<fr_db> db(new fr_db());
        db->ctx = c;
        db->K = (long long)K;
        db->ell = (int)ell;
        db->G = ((long long)K + n - 1) / n;
        db->tier = 4;
        db->schedule = 0;  // the stored diagonals are pre-rotated for the on-demand schedule
        const size_t ncts = (size_t)db->G * ell, lw = (size_t)level + 1;
        for (size_t e = 0; e < ncts; ++e)
            for (int t = 0; t < 2; ++t)
                for (int i = 0; i < L1; ++i) {
                    const u64 q = c->R.primes[i];
                    const uint64_t* p = cts + ((e * 2 + t) * lw + i) * N;
                    for (int x = 0; x < N; ++x)
                        if (p[x] >= q) raise(FR_ERR_FORMAT, "residue not below its prime");
                }
        db->bytes = ncts * 2 * L1 * (size_t)N * 8;
        if (c->budget && c->resident + db->bytes > c->budget)
            raise(FR_ERR_HBM_BUDGET, "database exceeds the HBM budget");
        if (!prerotated)  // the negative giant-step keys of the server-side pre-rotation
            for (long j = 1; j * (long)c->n1 < (long)ell; ++j) rot_key(c, frh::galois_of_rotation(c->R, -j * (long)c->n1));
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, db->bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            raise(e == cudaErrorMemoryAllocation ? FR_ERR_HBM_BUDGET : FR_ERR_CUDA,
                  std::string("cannot hold the encrypted diagonals: ") + cudaGetErrorString(e));
        }
        db->diags = (u64*)p;
        // limbs 0..L of both components, 64 ciphertexts per copy, then the NTT (into Montgomery
        // form when the enroller pre-rotated them)
        for (size_t e0 = 0; e0 < ncts; e0 += 64) {
            const size_t ne = std::min<size_t>(64, ncts - e0);
            u64* dst = db->diags + e0 * 2 * L1 * N;
            CU(cudaMemcpy2DAsync(dst, (size_t)L1 * N * 8, cts + e0 * 2 * lw * N, lw * N * 8, (size_t)L1 * N * 8, 2 * ne,
                                 cudaMemcpyHostToDevice, c->cur));
            if (prerotated) {
                PolyBatch pb{dst, (long long)L1 * N, L1, (int)(2 * ne * L1), pm_level(L)};
                launch_ntt_tomont(c->rd, pb, c->cur);
                c->launches++;
            } else {
                ntt(c, dst, (long long)L1 * N, L1, (int)(2 * ne * L1), pm_level(L), false);
            }
        }
        if (!prerotated) {
            // server-side pre-rotation (Eq. eq:prerotation on ciphertexts): diagonal j n1 + i,
            // j >= 1, is rotated by -j n1 with the negative giant-step key, 64 at a time into
            // scratch and copied back; then the whole database into Montgomery form
            const int n1 = (int)c->n1;
            const size_t cw1 = (size_t)2 * L1 * N;
            std::vector<size_t> todo;
            for (size_t e = 0; e < ncts; ++e)
                if ((int)(e % ell) >= n1) todo.push_back(e);
            Tmp rot(c, 64 * cw1);
            for (size_t t0 = 0; t0 < todo.size(); t0 += 64) {
                const size_t nt = std::min<size_t>(64, todo.size() - t0);
                std::vector<KSReq> reqs;
                for (size_t t = 0; t < nt; ++t) {
                    const size_t e = todo[t0 + t];
                    const long j = (long)(e % ell) / n1;
                    const u64 gk = frh::galois_of_rotation(c->R, -j * n1);
                    const u64* src = db->diags + e * cw1;
                    reqs.push_back(KSReq{src + (size_t)L1 * N, rot_key(c, gk), (u32)gk, 1, src, L1, rot.p + t * cw1, L1});
                }
                keyswitch(c, L, reqs);
                for (size_t t = 0; t < nt; ++t) copy_d2d(c, db->diags + todo[t0 + t] * cw1, rot.p + t * cw1, cw1);
            }
            launch_to_mont(db->diags, N, pm_level(L), c->d_primes, (long long)(ncts * cw1), c->cur);
            c->launches++;
        }
        CU(cudaStreamSynchronize(c->cur));
        c->resident += db->bytes;
        c->dbs.insert(db.get());
        *out = db.release();
    });
}

fr_status fr_db_info(const fr_db* db, uint32_t* tier, uint64_t* groups, uint64_t* bytes, uint32_t* schedule) {
    if (!db) return FR_ERR_INVALID_ARG;
    if (schedule) *schedule = (uint32_t)db->schedule;
    if (tier) *tier = (uint32_t)db->tier;
    if (groups) *groups = (uint64_t)db->G;
    if (bytes) *bytes = (uint64_t)db->bytes;
    return FR_OK;
}

void fr_free_db(fr_db* db) {
    if (!db) return;
    if (!db->ctx) {  // its context was freed first, with the device memory
        delete db;
        return;
    }
    db->ctx->dbs.erase(db);
    if (db->ctx) serve_drain_db(db->ctx, db);
    if (db->ctx) drop_graphs(db->ctx, db);
    if (db->ctx) {
        cudaStreamSynchronize(db->ctx->stream);
        db->ctx->resident -= db->bytes;
    }
    cudaFree(db->diags);
    cudaFree(db->templates);
    cudaFree(db->coeffs);
    delete db;
}

static fr_status encrypt_slots(const fr_ctx* c, const fr_keys* k, const std::vector<double>& z, uint64_t seed,
                               fr_ct** out) {
    return guard([&] {
        std::unique_ptr<fr_ct> ct(new fr_ct());
        ct->ctx = c;
        ct->level = c->R.nq - 1;
        ct->cap = c->R.nq;
        ct->scale = std::ldexp(1.0, c->R.scale_bits);
        ct->host.resize((size_t)2 * c->R.nq * c->R.N);
        frh::encrypt(c->R, k->ks, z.data(), seed, ct->host.data());
        *out = ct.release();
    });
}

fr_status fr_encrypt(const fr_ctx* c, const fr_keys* k, const double* q, size_t ell, uint64_t seed, fr_ct** out) {
    if (!c || !k || !q || !out) {
        g_last_error = "null argument";
        return FR_ERR_INVALID_ARG;
    }
    const size_t n = (size_t)c->R.N / 2;
    if (ell == 0 || n % ell != 0) {
        g_last_error = "ell must divide N/2";
        return FR_ERR_INVALID_ARG;
    }
    std::vector<double> z(n);
    for (size_t i = 0; i < n; ++i) z[i] = q[i % ell];
    return encrypt_slots(c, k, z, seed, out);
}

fr_status fr_encrypt_slots(const fr_ctx* c, const fr_keys* k, const double* zin, size_t n, uint64_t seed,
                           fr_ct** out) {
    if (!c || !k || !zin || !out || n != (size_t)c->R.N / 2) {
        g_last_error = "bad arguments (need N/2 slot values)";
        return FR_ERR_INVALID_ARG;
    }
    std::vector<double> z(zin, zin + n);
    return encrypt_slots(c, k, z, seed, out);
}

fr_status fr_ct_import(const fr_ctx* c, const uint64_t* buf, uint32_t level, double scale, fr_ct** out) {
    return guard([&] {
        if (!c || !buf || !out) raise(FR_ERR_INVALID_ARG, "null argument");
        if ((int)level >= c->R.nq) raise(FR_ERR_LEVEL, "level out of range");
        const size_t N = c->R.N, L1 = level + 1;
        for (int t = 0; t < 2; ++t)
            for (size_t i = 0; i < L1; ++i) {
                const u64 q = c->R.primes[i];
                const uint64_t* p = buf + (t * L1 + i) * N;
                for (size_t k = 0; k < N; ++k)
                    if (p[k] >= q) raise(FR_ERR_FORMAT, "residue not below its prime");
            }
        std::unique_ptr<fr_ct> ct(new fr_ct());
        ct->ctx = c;
        ct->level = (int)level;
        ct->cap = (int)L1;
        ct->scale = scale;
        ct->host.assign(buf, buf + 2 * L1 * N);
        *out = ct.release();
    });
}

fr_status fr_ct_export(const fr_ct* ct, uint64_t* buf, size_t words, uint32_t* level, double* scale) {
    return guard([&] {
        if (!ct || !buf) raise(FR_ERR_INVALID_ARG, "null argument");
        fr_ctx* c = const_cast<fr_ctx*>(ct->ctx);
        if (!c) raise(FR_ERR_INVALID_ARG, "ciphertext without context");
        const size_t need = (size_t)2 * (ct->level + 1) * c->R.N;
        if (words < need) raise(FR_ERR_INVALID_ARG, "export buffer too small");
        export_words(c, ct, buf);
        if (level) *level = (uint32_t)ct->level;
        if (scale) *scale = ct->scale;
    });
}

fr_status fr_ct_info(const fr_ct* ct, uint32_t* level, int* on_device) {
    if (!ct) return FR_ERR_INVALID_ARG;
    if (level) *level = (uint32_t)ct->level;
    if (on_device) *on_device = ct->on_dev ? 1 : 0;
    return FR_OK;
}

fr_status fr_ct_upload(fr_ctx* c, fr_ct* ct) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        check_ct(c, ct);
        if (ct->on_dev) return;
        const int cap = ct->level + 1;
        auto blk = new_block(c, ctw(c, cap));
        to_device(c, ct, blk->p, cap);
        CU(cudaStreamSynchronize(c->cur));
        ct->block = blk;
        ct->dev = blk->p;
        ct->cap = cap;
        ct->on_dev = true;
        ct->host.clear();
        ct->host.shrink_to_fit();
    });
}

void fr_free_ct(fr_ct* ct) { delete ct; }
void fr_free_cts(fr_ct** cts, size_t n) {
    if (!cts) return;
    for (size_t i = 0; i < n; ++i) delete cts[i];
    delete[] cts;
}

fr_status fr_decrypt(const fr_ctx* c, const fr_keys* k, const fr_ct* ct, double* slots, size_t n_slots) {
    return guard([&] {
        if (!c || !k || !ct || !slots) raise(FR_ERR_INVALID_ARG, "null argument");
        check_ct(c, ct);
        const int N = c->R.N;
        std::vector<u64> w((size_t)2 * (ct->level + 1) * N);
        export_words(const_cast<fr_ctx*>(c), ct, w.data());
        std::vector<double> x(N);
        frh::decrypt_values(c->R, k->ks, w.data(), ct->level, x.data());
        std::vector<double> z(N / 2);
        frh::decode_values(c->R, x.data(), ct->scale, z.data());
        for (size_t i = 0; i < n_slots && i < z.size(); ++i) slots[i] = z[i];
    });
}

// ---------------------------------------------------------------------------
// primitives on device ciphertexts
// ---------------------------------------------------------------------------
static const u64* dev_view(fr_ctx* c, const fr_ct* ct, std::unique_ptr<Tmp>& hold, int* cap) {
    if (ct->on_dev) {
        *cap = ct->cap;
        return ct->dev;
    }
    hold.reset(new Tmp(c, ctw(c, ct->level + 1)));
    to_device(c, ct, hold->p, ct->level + 1);
    *cap = ct->level + 1;
    return hold->p;
}

fr_status fr_rotate_hoisted(fr_ctx* c, const fr_ct* ct, const int32_t* ks, size_t n, fr_ct** out) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        check_ct(c, ct);
        if (!ks || !out || n == 0) raise(FR_ERR_INVALID_ARG, "null argument");
        CU(cudaSetDevice(c->device));
        std::unique_ptr<Tmp> hold;
        int cap;
        const u64* src = dev_view(c, ct, hold, &cap);
        const int l = ct->level, L1 = l + 1;
        auto blk = new_block(c, n * ctw(c, L1));
        std::vector<long> kv(ks, ks + n);
        std::vector<u64*> outs;
        for (size_t i = 0; i < n; ++i) outs.push_back(blk->p + i * ctw(c, L1));
        rotate_cts(c, l, {src}, cap, kv, outs, L1, true);
        for (size_t i = 0; i < n; ++i) out[i] = new_dev_ct(c, blk, outs[i], l, L1);
    });
}

fr_status fr_rotate(fr_ctx* c, const fr_ct* ct, int32_t k, fr_ct** out) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        check_ct(c, ct);
        if (!out) raise(FR_ERR_INVALID_ARG, "null argument");
        CU(cudaSetDevice(c->device));
        std::unique_ptr<Tmp> hold;
        int cap;
        const u64* src = dev_view(c, ct, hold, &cap);
        const int l = ct->level, L1 = l + 1;
        auto blk = new_block(c, ctw(c, L1));
        rotate_cts(c, l, {src}, cap, {(long)k}, {blk->p}, L1, false);
        *out = new_dev_ct(c, blk, blk->p, l, L1);
    });
}

fr_status fr_rescale(fr_ctx* c, const fr_ct* ct, fr_ct** out) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        check_ct(c, ct);
        if (!out) raise(FR_ERR_INVALID_ARG, "null argument");
        if (ct->level < 1) raise(FR_ERR_LEVEL, "cannot rescale at level 0");
        CU(cudaSetDevice(c->device));
        std::unique_ptr<Tmp> hold;
        int cap;
        const u64* src = dev_view(c, ct, hold, &cap);
        const int l = ct->level;
        auto blk = new_block(c, ctw(c, l));
        rescale(c, src, 1, l, cap, blk->p, l);
        *out = new_dev_ct(c, blk, blk->p, l - 1, l);
    });
}

fr_status fr_mul_relin(fr_ctx* c, const fr_ct* a, const fr_ct* b, fr_ct** out) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        check_ct(c, a);
        check_ct(c, b);
        if (!out) raise(FR_ERR_INVALID_ARG, "null argument");
        if (a->level != b->level) raise(FR_ERR_LEVEL, "operands at different levels");
        CU(cudaSetDevice(c->device));
        std::unique_ptr<Tmp> ha, hb;
        int ca, cb;
        const u64* pa = dev_view(c, a, ha, &ca);
        const u64* pb = dev_view(c, b, hb, &cb);
        const int l = a->level, L1 = l + 1;
        auto blk = new_block(c, ctw(c, L1));
        mul_relin(c, l, {pa}, ca, {pb}, cb, {blk->p}, L1);
        *out = new_dev_ct(c, blk, blk->p, l, L1);
    });
}

fr_status fr_add(fr_ctx* c, const fr_ct* a, const fr_ct* b, fr_ct** out) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        check_ct(c, a);
        check_ct(c, b);
        if (!out) raise(FR_ERR_INVALID_ARG, "null argument");
        CU(cudaSetDevice(c->device));
        std::unique_ptr<Tmp> ha, hb;
        int ca, cb;
        const u64* pa = dev_view(c, a, ha, &ca);
        const u64* pb = dev_view(c, b, hb, &cb);
        const int l = std::min(a->level, b->level), L1 = l + 1;
        auto blk = new_block(c, ctw(c, L1));
        add_cts(c, pa, ca, 0, pb, cb, 0, blk->p, L1, 0, l, 1);
        *out = new_dev_ct(c, blk, blk->p, l, L1);
    });
}

fr_status fr_chebyshev(fr_ctx* c, const fr_ct* ct, fr_ct** out) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        check_ct(c, ct);
        if (!out) raise(FR_ERR_INVALID_ARG, "null argument");
        if (c->cheb_n == 0) raise(FR_ERR_INVALID_ARG, "context has no Chebyshev degree");
        CU(cudaSetDevice(c->device));
        std::unique_ptr<Tmp> hold;
        int cap;
        const u64* src = dev_view(c, ct, hold, &cap);
        const int lo = ct->level - c->cmp_depth;
        if (lo < 0) raise(FR_ERR_LEVEL, "not enough levels for the threshold");
        auto blk = new_block(c, ctw(c, lo + 1));
        threshold(c, src, 1, ct->level, cap, blk->p, lo + 1);
        *out = new_dev_ct(c, blk, blk->p, lo, lo + 1);
    });
}

// Membership tail over threshold ciphertexts that come from several places (the groups of a
// database split across processes): the mod-q sum of all parts, then RotateAndSum over all slots
// (Algorithm 5's aggregation). Parts must share one level. With the FR_MODE_IDENTIFY outputs of
// every group as parts, the result equals FR_MODE_MEMBERSHIP on the whole database bit for bit:
// the sum is exact and independent of the order of its terms.
fr_status fr_membership_reduce(fr_ctx* c, const fr_ct* const* parts, size_t n, fr_ct** out) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        if (!parts || !out || n == 0) raise(FR_ERR_INVALID_ARG, "null argument or no parts");
        for (size_t i = 0; i < n; ++i) {
            check_ct(c, parts[i]);
            if (parts[i]->level != parts[0]->level) raise(FR_ERR_LEVEL, "parts at different levels");
        }
        CU(cudaSetDevice(c->device));
        const int l = parts[0]->level, L1 = l + 1;
        const size_t cw = (size_t)ctw(c, L1);
        Tmp stage(c, n * cw);
        for (size_t i = 0; i < n; ++i) to_device(c, parts[i], stage.p + i * cw, L1);
        auto blk = new_block(c, cw);
        launch_sum(stage.p, L1, (long long)cw, (int)n, blk->p, L1, l, c->d_primes, c->R.N, c->cur);
        c->launches++;
        rotate_sum(c, blk->p, L1, l);
        *out = new_dev_ct(c, blk, blk->p, l, L1);
    });
}

fr_status fr_rotate_sum(fr_ctx* c, const fr_ct* ct, fr_ct** out) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        check_ct(c, ct);
        if (!out) raise(FR_ERR_INVALID_ARG, "null argument");
        CU(cudaSetDevice(c->device));
        const int l = ct->level, L1 = l + 1;
        auto blk = new_block(c, ctw(c, L1));
        to_device(c, ct, blk->p, L1);
        rotate_sum(c, blk->p, L1, l);
        *out = new_dev_ct(c, blk, blk->p, l, L1);
    });
}

// ---------------------------------------------------------------------------
// The encrypted 1:N match: on-demand BSGS with hoisted baby steps and
// pre-rotated diagonals (Algorithms 5 and 6; Eq. eq:prerotation), then the
// Chebyshev threshold and, for membership, the group sum and RotateAndSum.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

// shapes of the match outputs per query: count and level
void match_shape(const fr_ctx* c, const fr_db* db, fr_mode mode, int* nout, int* lo) {
    const int L = c->work_level;
    if (mode == FR_MODE_SCORES) {
        *nout = (int)db->G;
        *lo = L - 1;
    } else {
        *nout = mode == FR_MODE_IDENTIFY ? (int)db->G : 1;
        *lo = L - 1 - c->cmp_depth;
    }
}

// A batch: query b matches database dbs[b]; its score ciphertexts are S + soff[b] (in
// ciphertexts of 2 L limb-polys), soff[B] the total.
struct BatchPlan {
    std::vector<const fr_db*> dbs;
    std::vector<long long> soff;
    explicit BatchPlan(const std::vector<const fr_db*>& d) : dbs(d), soff(d.size() + 1, 0) {
        for (size_t b = 0; b < d.size(); ++b) soff[b + 1] = soff[b] + d[b]->G;
    }
};

// S2-S5 by the on-demand schedule for the queries qs of a batch (q: [B][2][L+1][N], evaluation
// form, level = work level): their scores at level L-1 into S per the plan. Every stage runs
// once for these queries: one ModUp per query, key-grouped inner products; then group by group
// (over the queries whose database has that group) one MAC per query, one rescale, the giant
// rotations with each key read once, the sums. A database encoded per query (tiers B, C) is
// encoded once per group for all its queries.
void ondemand_scores(fr_ctx* c, const BatchPlan& P, const u64* q, const std::vector<int>& qs, u64* S) {
    const int L = c->work_level;
    const int N = c->R.N, n1 = (int)c->n1, ell = (int)c->ell;
    const int n2 = (ell + n1 - 1) / n1;
    const int L1 = L + 1;
    const int B = (int)qs.size();
    const size_t cw1 = (size_t)ctw(c, L1), cw = (size_t)ctw(c, L);
    // baby steps in Q_l u P (double hoisting): babies and diagonals span every position of Q_l u P
    const bool pq = c->hoist_babies;
    const int npos = L1 + c->R.np;
    const int nlx = pq ? npos : L1;                       // limbs of a baby ct and of a diagonal
    const size_t bw = (size_t)2 * nlx * N;                // words of one baby
    const DevPrime* mprimes = pq ? primes_ext(c, L) : c->d_primes;
    if (pq)
        for (int b = 0; b < B; ++b)
            if (P.dbs[qs[b]]->tier == 4)
                raise(FR_ERR_UNSUPPORTED, "encrypted databases need hoist_babies = 0");
    // S2: baby steps B_{b,i} = Rot_i(q_b), hoisted per query
    std::unique_ptr<Prof> stage(new Prof(c, "stage:babies"));
    Tmp babies(c, (size_t)B * n1 * bw);  // [B][n1][2][nlx][N]
    if (!pq) {
        for (int b = 0; b < B; ++b) copy_d2d(c, babies.p + (size_t)b * n1 * cw1, q + (size_t)qs[b] * cw1, cw1);
        if (n1 > 1) {
            std::vector<KSReq> reqs;
            for (int b = 0; b < B; ++b) {
                u64* q0 = babies.p + (size_t)b * n1 * cw1;
                for (int i = 1; i < n1; ++i) {
                    const u64 g = frh::galois_of_rotation(c->R, i);
                    reqs.push_back(KSReq{q0 + (size_t)L1 * N, rot_key(c, g), (u32)g, 1, q0, L1, q0 + (size_t)i * cw1, L1});
                }
            }
            keyswitch(c, L, reqs);
        }
    } else {
        // one ModUp per query; the inner products of babies 1..n1-1 land in the babies buffer;
        // then P sigma_i(q.b) on their Q positions and baby 0 = P q
        if (n1 > 1) {
            std::vector<KSReq> reqs;
            for (int b = 0; b < B; ++b) {
                const u64* qb = q + (size_t)qs[b] * cw1;
                for (int i = 1; i < n1; ++i) {
                    const u64 g = frh::galois_of_rotation(c->R, i);
                    reqs.push_back(KSReq{qb + (size_t)L1 * N, rot_key(c, g), (u32)g, 1, qb, L1,
                                         babies.p + ((size_t)b * n1 + i) * bw, npos});
                }
            }
            const int beta = c->R.digits_at(L);
            modup_chunks(c, L, reqs, [&](const std::vector<const KSReq*>& rq, const std::vector<const u64*>& ex) {
                IPJobs ij;
                ij.ngroups = 0;
                const int nj = (int)rq.size();
                for (int j = 0; j < nj; ++j) {
                    ij.j[j] = IPJob{ex[j], rq[j]->key, rq[j]->out, rq[j]->galois, 0, rq[j]->add};  // + P sigma(b)
                    if (j == 0 || rq[j]->key != rq[j - 1]->key) {
                        ij.gkey[ij.ngroups] = rq[j]->key;
                        ij.gstart[ij.ngroups] = j;
                        ij.ngroups++;
                    }
                }
                ij.gstart[ij.ngroups] = nj;
                Prof p(c, "ip", 8.0 * N * npos * (ij.ngroups * 2.0 * beta + nj * (double)beta + nj * 2.0) +
                                    8.0 * N * nj * L1);
                launch_ip(ij, beta, npos, L, c->key_level + 1, c->key_limbs, c->d_primes, pm_ext(c, L), c->R.logN,
                          c->cur, c->d_pmod, c->d_pmod_s);
                c->launches++;
            });
        }
        // baby 0 = P q; queries are gathered in qs order and their inputs sit at q + qs[b] cw1:
        // one launch per run of consecutive indices
        for (int b0 = 0; b0 < B;) {
            int b1 = b0 + 1;
            while (b1 < B && qs[b1] == qs[b1 - 1] + 1) ++b1;
            Prof p(c, "misc", 8.0 * N * (b1 - b0) * 2.0 * (npos + L1));
            launch_baby0_pq(babies.p + (size_t)b0 * n1 * bw, (long long)n1 * bw, q + (size_t)qs[b0] * cw1, (long long)cw1,
                            L1, b1 - b0, npos, L, mprimes, c->d_pmod, c->d_pmod_s, N, c->cur);
            c->launches++;
            b0 = b1;
        }
    }
    // S3-S5 group by group: (tiers B, C: encode the group's diagonals), MAC, rescale, giant
    // rotations, sum; at most 8 databases encoded per query in flight
    stage.reset();
    long long Gmax = 0;
    for (int b = 0; b < B; ++b) Gmax = std::max(Gmax, P.dbs[qs[b]]->G);
    for (long long g = 0; g < Gmax; ++g) {
        std::vector<int> sel;  // positions in qs of the queries whose database has group g
        for (int b = 0; b < B; ++b)
            if (g < P.dbs[qs[b]]->G) sel.push_back(b);
        for (size_t s0 = 0; s0 < sel.size();) {
            std::vector<const fr_db*> enc;  // databases encoded for this chunk
            size_t s1 = s0;
            for (; s1 < sel.size(); ++s1) {
                const fr_db* d = P.dbs[qs[sel[s1]]];
                if (d->tier == 1 || d->tier == 4 || std::find(enc.begin(), enc.end(), d) != enc.end()) continue;
                if (enc.size() == 8) break;
                enc.push_back(d);
            }
            const int nb = (int)(s1 - s0);
            std::unique_ptr<Tmp> dg;
            if (!enc.empty()) {
                stage.reset(new Prof(c, "stage:encode"));
                dg.reset(new Tmp(c, enc.size() * (size_t)ell * nlx * N));
                for (size_t e = 0; e < enc.size(); ++e) {
                    u64* dst = dg->p + e * (size_t)ell * nlx * N;
                    if (enc[e]->tier == 2) encode_group(c, enc[e]->templates, enc[e]->K, g, dst, (int)c->n1, nlx);
                    else expand_group(c, enc[e]->coeffs + (size_t)g * ell * N, dst, nlx);
                }
            }
            auto diag_of = [&](const fr_db* d) -> const u64* {
                if (d->tier == 1) return d->diags + (size_t)g * ell * d->nl * N;
                if (d->tier == 4) return d->diags + (size_t)g * ell * 2 * L1 * N;
                const size_t e = std::find(enc.begin(), enc.end(), d) - enc.begin();
                return dg->p + e * (size_t)ell * nlx * N;
            };
            stage.reset(new Prof(c, "stage:mac"));
            Tmp Pj(c, (size_t)nb * n2 * bw);  // [nb][n2][2][nlx][N]
            int nenc = 0;  // queries of the chunk against encrypted databases
            for (int t = 0; t < nb; ++t) nenc += P.dbs[qs[sel[s0 + t]]]->tier == 4;
            std::unique_ptr<Tmp> D3;  // their unrelinearised products, [nenc][n2][3][L1][N]
            if (nenc) D3.reset(new Tmp(c, (size_t)nenc * n2 * 3 * L1 * N));
            std::vector<KSReq> relin;
            for (int t = 0, e = 0; t < nb; ++t) {
                const int b = sel[s0 + t];
                const fr_db* d = P.dbs[qs[b]];
                // up to 4 queries against the same diagonals (consecutive babies) share one launch
                // that reads each diagonal word once for all of them: the persistent pipeline
                // k_mac_ring where its tiling fits, else k_mac_pipe. A single query runs k_mac
                // below (measured faster for one query: 0.98 ms against 1.13 ms at the headline)
                int cnt = 1;
                if (d->tier != 4 && (mac_ring_fits(n1, ell, N, 2) || mac_pipe_fits(n1, ell, N)))
                    while (cnt < 4 && t + cnt < nb && sel[s0 + t + cnt] == b + cnt &&
                           diag_of(P.dbs[qs[b + cnt]]) == diag_of(d))
                        ++cnt;
                if (d->tier != 4 && cnt > 1 && mac_ring_fits(n1, ell, N, cnt)) {
                    Prof p(c, "mac", 8.0 * N * nlx * ((double)ell + cnt * (2.0 * n1 + 2.0 * n2)));
                    launch_mac_ring(babies.p + (size_t)b * n1 * bw, (long long)n1 * bw, nlx, diag_of(d),
                                    Pj.p + (size_t)t * n2 * bw, (long long)n2 * bw, nlx, nlx, n1, ell, cnt, mprimes, N,
                                    c->cur);
                    c->launches++;
                    t += cnt - 1;
                    continue;
                }
                if (cnt > 1 && mac_pipe_fits(n1, ell, N)) {
                    Prof p(c, "mac", 8.0 * N * nlx * ((double)ell + cnt * (2.0 * n1 + 2.0 * n2)));
                    launch_mac_pipe(babies.p + (size_t)b * n1 * bw, (long long)n1 * bw, nlx, diag_of(d),
                                    Pj.p + (size_t)t * n2 * bw, (long long)n2 * bw, nlx, nlx, n1, ell, cnt, mprimes, N,
                                    c->cur);
                    c->launches++;
                    t += cnt - 1;
                    continue;
                }
                if (d->tier == 4) {
                    // ct x ct products summed per giant step; one relinearisation each (below)
                    u64* o = D3->p + (size_t)e++ * n2 * 3 * L1 * N;
                    Prof p(c, "mac", 8.0 * N * L1 * (2.0 * ell + 2.0 * n1 + 3.0 * n2));
                    launch_mac_ct(babies.p + (size_t)b * n1 * cw1, L1, diag_of(d), o, L1, L1, n1, n2, ell, c->d_primes,
                                  N, c->cur);
                    c->launches++;
                    for (int j = 0; j < n2; ++j) {
                        const u64* dj = o + (size_t)j * 3 * L1 * N;
                        relin.push_back(KSReq{dj + (size_t)2 * L1 * N, relin_key(c), 1u, 2, dj, L1,
                                              Pj.p + ((size_t)t * n2 + j) * cw1, L1});
                    }
                    continue;
                }
                Prof p(c, "mac", 8.0 * N * nlx * ((double)ell + 2.0 * n1 + 2.0 * n2));
                launch_mac(babies.p + (size_t)b * n1 * bw, (long long)n1 * bw, nlx, diag_of(d),
                           Pj.p + (size_t)t * n2 * bw, (long long)n2 * bw, nlx, nlx, n1, n2, ell, 1, mprimes, N, c->cur);
                c->launches++;
            }
            if (!relin.empty()) {
                stage.reset(new Prof(c, "stage:relin"));
                keyswitch(c, L, relin);
            }
            Tmp Gs(c, (size_t)nb * n2 * cw);  // [nb][n2][2][L][N]
            if (pq)
                moddown_rescale(c, L, Pj.p, nullptr, nb * n2, Gs.p, L, (long long)cw, RescaleEpi());
            else
                rescale(c, Pj.p, nb * n2, L, L1, Gs.p, L);
            stage.reset(new Prof(c, "stage:giants"));
            if (n2 > 1 && c->hoist_giants) {
                // S = P_0 + sum_j Rot_{j n1}(P_j) with one ModDown per (query, group)
                std::vector<KSReq> reqs;
                std::vector<const u64*> base;
                std::vector<u64*> outp;
                for (int t = 0; t < nb; ++t) {
                    base.push_back(Gs.p + (size_t)t * n2 * cw);
                    outp.push_back(S + ((size_t)P.soff[qs[sel[s0 + t]]] + g) * cw);
                }
                for (int j = 1; j < n2; ++j) {
                    const u64 gk = frh::galois_of_rotation(c->R, (long)j * n1);
                    const u64* key = rot_key(c, gk);
                    for (int t = 0; t < nb; ++t) {
                        const u64* src = Gs.p + ((size_t)t * n2 + j) * cw;
                        KSReq r{src + (size_t)L * N, key, (u32)gk, 1, src, L, nullptr, L};
                        r.sum_dst = t;
                        reqs.push_back(r);
                    }
                }
                keyswitch_sums(c, L - 1, reqs, base, L, outp, L);
                stage.reset();
                s0 = s1;
                continue;
            }
            if (n2 > 1) {
                Tmp Pr(c, (size_t)nb * n2 * cw);
                copy_d2d(c, Pr.p, Gs.p, (size_t)nb * n2 * cw);
                std::vector<KSReq> reqs;
                for (int j = 1; j < n2; ++j) {
                    const u64 gk = frh::galois_of_rotation(c->R, (long)j * n1);
                    const u64* key = rot_key(c, gk);
                    for (int t = 0; t < nb; ++t) {
                        const u64* src = Pr.p + ((size_t)t * n2 + j) * cw;
                        reqs.push_back(KSReq{src + (size_t)L * N, key, (u32)gk, 1, src, L,
                                             Gs.p + ((size_t)t * n2 + j) * cw, L});
                    }
                }
                keyswitch(c, L - 1, reqs);
            }
            for (int t = 0; t < nb; ++t) {
                const int b = sel[s0 + t];
                Prof p(c, "misc", 8.0 * N * 2.0 * L * (n2 + 1));
                launch_sum(Gs.p + (size_t)t * n2 * cw, L, cw, n2, S + ((size_t)P.soff[qs[b]] + g) * cw, L, L - 1,
                           c->d_primes, N, c->cur);
                c->launches++;
            }
            stage.reset();
            s0 = s1;
        }
    }
}

// S2-S5 by the rotated-query table of Algorithm 1 for one query q ([2][L+1][N], evaluation
// form, level = work level): rotQ[i] = Rot_i(q) for i < n1, hoisted over one ModUp of q;
// rotQ[j n1 + i] = Rot_{j n1}(rotQ[i]), hoisted over one ModUp per baby (the key switch
// shares the ModUp of equal inputs); then S_g = Rescale(sum_{m < ell} rotQ[m] (.) D_{g,m})
// with plain diagonals, for every group, into S [G][2][L][N] at level L-1.
void table_scores(fr_ctx* c, const fr_db* db, const u64* q, u64* S) {
    const int L = c->work_level, L1 = L + 1;
    const int N = c->R.N, n1 = (int)c->n1, ell = (int)c->ell;
    const int n2 = (ell + n1 - 1) / n1;
    const long long G = db->G;
    const size_t cw1 = (size_t)ctw(c, L1), cw = (size_t)ctw(c, L);
    std::unique_ptr<Prof> stage(new Prof(c, "stage:babies"));
    Tmp tab(c, (size_t)ell * cw1);  // [ell][2][L1][N]
    copy_d2d(c, tab.p, q, cw1);
    std::vector<KSReq> reqs;
    for (int i = 1; i < n1; ++i) {
        const u64 g = frh::galois_of_rotation(c->R, i);
        reqs.push_back(KSReq{tab.p + (size_t)L1 * N, rot_key(c, g), (u32)g, 1, tab.p, L1, tab.p + (size_t)i * cw1, L1});
    }
    keyswitch(c, L, reqs);
    stage.reset(new Prof(c, "stage:giants"));
    reqs.clear();
    for (int j = 1; j < n2; ++j) {
        const u64 gk = frh::galois_of_rotation(c->R, (long)j * n1);
        const u64* key = rot_key(c, gk);
        for (int i = 0; i < n1 && j * n1 + i < ell; ++i) {
            const u64* src = tab.p + (size_t)i * cw1;
            reqs.push_back(KSReq{src + (size_t)L1 * N, key, (u32)gk, 1, src, L1, tab.p + (size_t)(j * n1 + i) * cw1, L1});
        }
    }
    keyswitch(c, L, reqs);
    // step 4: groups in chunks (tier C encodes a chunk of groups per pass)
    const long long GC = db->tier != 1 ? std::min<long long>(G, 8) : G;
    std::unique_ptr<Tmp> dg;
    if (db->tier != 1) dg.reset(new Tmp(c, (size_t)GC * ell * L1 * N));
    for (long long g0 = 0; g0 < G; g0 += GC) {
        const int gc = (int)std::min<long long>(GC, G - g0);
        const u64* D = db->diags + (size_t)g0 * ell * L1 * N;
        if (db->tier == 2) {
            stage.reset(new Prof(c, "stage:encode"));
            for (int t = 0; t < gc; ++t)
                encode_group(c, db->templates, db->K, g0 + t, dg->p + (size_t)t * ell * L1 * N, ell, L1);
            D = dg->p;
        } else if (db->tier == 3) {
            stage.reset(new Prof(c, "stage:encode"));
            for (int t = 0; t < gc; ++t)
                expand_group(c, db->coeffs + (size_t)(g0 + t) * ell * N, dg->p + (size_t)t * ell * L1 * N, L1);
            D = dg->p;
        }
        stage.reset(new Prof(c, "stage:mac"));
        Tmp Pt(c, (size_t)gc * cw1);
        {
            const int GG = gc >= 8 ? 8 : gc >= 4 ? 4 : gc >= 2 ? 2 : 1;
            Prof p(c, "mac", 8.0 * N * L1 * ((double)ell * gc + 2.0 * ell * ((gc + GG - 1) / GG) + 2.0 * gc));
            launch_mac_table(tab.p, L1, D, (long long)ell * L1 * N, gc, Pt.p, L1, (long long)cw1, L1, ell, c->d_primes,
                             N, c->cur);
            c->launches++;
        }
        rescale(c, Pt.p, gc, L, L1, S + (size_t)g0 * cw, L);
        stage.reset();
    }
}

// The whole match for B queries already in HBM (q: [B][2][L+1][N], evaluation form,
// level = work level), query b against dbs[b]; writes each query's output ciphertexts
// (cap = level + 1) contiguously to out, query after query.
void match_pipeline(fr_ctx* c, const std::vector<const fr_db*>& dbs, const u64* q, fr_mode mode, u64* out) {
    const int L = c->work_level, N = c->R.N;
    const int B = (int)dbs.size();
    const BatchPlan P(dbs);
    const long long total = P.soff[B];
    const size_t cw1 = (size_t)ctw(c, L + 1), cw = (size_t)ctw(c, L);
    const bool scores_only = mode == FR_MODE_SCORES;
    Tmp sbuf(c, scores_only ? 1 : (size_t)total * cw);
    u64* S = scores_only ? out : sbuf.p;  // scores of query b from S + soff[b] cw
    std::vector<int> od;
    for (int b = 0; b < B; ++b) {
        if (dbs[b]->schedule == 1) table_scores(c, dbs[b], q + (size_t)b * cw1, S + (size_t)P.soff[b] * cw);
        else od.push_back(b);
    }
    if (!od.empty()) ondemand_scores(c, P, q, od, S);
    std::unique_ptr<Prof> stage;
    if (scores_only) {
        CU(cudaGetLastError());  // a launch the device refused (configuration, resources) fails the match
        return;
    }
    // S6: threshold on every (query, group) score ciphertext (batched)
    const int lo = L - 1 - c->cmp_depth;
    const size_t cwo = (size_t)ctw(c, lo + 1);
    if (mode == FR_MODE_IDENTIFY) {
        stage.reset(new Prof(c, "stage:cheb"));
        threshold(c, S, (int)total, L - 1, L, out, lo + 1);
        CU(cudaGetLastError());  // a launch the device refused (configuration, resources) fails the match
        return;
    }
    Tmp cbuf(c, (size_t)total * cwo);
    stage.reset(new Prof(c, "stage:cheb"));
    threshold(c, S, (int)total, L - 1, L, cbuf.p, lo + 1);
    // S7: per query, sum over its groups, then RotateAndSum over all slots
    stage.reset(new Prof(c, "stage:sum"));
    for (int b = 0; b < B; ++b) {
        Prof p(c, "misc");
        launch_sum(cbuf.p + (size_t)P.soff[b] * cwo, lo + 1, cwo, (int)dbs[b]->G, out + (size_t)b * cwo, lo + 1, lo,
                   c->d_primes, N, c->cur);
        c->launches++;
    }
    rotate_sum(c, out, lo + 1, lo, B);
    CU(cudaGetLastError());  // a launch the device refused (configuration, resources) fails the match
}

// Number of output ciphertexts of a batch and the offset of each query's first output.
long long match_outputs(const std::vector<const fr_db*>& dbs, fr_mode mode, std::vector<long long>& first) {
    first.assign(dbs.size() + 1, 0);
    for (size_t b = 0; b < dbs.size(); ++b) first[b + 1] = first[b] + (mode == FR_MODE_MEMBERSHIP ? 1 : dbs[b]->G);
    return first.back();
}

}  // namespace

// A match replayed as a CUDA graph: queries staged in `in`, outputs left in `out`.
struct MatchGraph {
    cudaGraphExec_t exec = nullptr;
    u64* in = nullptr;
    u64* out = nullptr;
    int runs = 0;
    uint64_t kernels = 0;
};

namespace {
std::mutex g_graph_mu;
// key: context, the database of each query, mode
std::map<std::tuple<const fr_ctx*, std::vector<const fr_db*>, int>, MatchGraph> g_graphs;

void drop_graphs(const fr_ctx* c, const fr_db* db) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
        const auto& v = std::get<1>(it->first);
        if (std::get<0>(it->first) == c && (db == nullptr || std::find(v.begin(), v.end(), db) != v.end())) {
            if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
            cudaFree(it->second.in);
            cudaFree(it->second.out);
            it = g_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

// B queries, query b against dbs[b]: validate, stage, run (eagerly, or as a CUDA graph from
// the second call with the same context, databases and mode on), return the output handles,
// query after query.
void match_queries(fr_ctx* c, const std::vector<const fr_db*>& dbs, const fr_ct* const* queries, fr_mode mode,
                   fr_ct*** out, size_t* n_out) {
    need_device(c);
    std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
    const int B = (int)dbs.size();
    if (!queries || !out || !n_out || B < 1) raise(FR_ERR_INVALID_ARG, "null argument or empty batch");
    for (int b = 0; b < B; ++b) {
        if (!dbs[b]) raise(FR_ERR_INVALID_ARG, "null database");
        if (dbs[b]->ctx != c) raise(FR_ERR_INVALID_ARG, "database belongs to another context");
        check_ct(c, queries[b]);
        if (queries[b]->level != c->R.nq - 1) raise(FR_ERR_LEVEL, "queries must be at the top level");
    }
    const int L = c->work_level;
    if ((size_t)c->n1 * 2 * 16 * 8 > (128u << 10))
        raise(FR_ERR_UNSUPPORTED, "n1 too large for the MAC's shared-memory staging of the baby steps");
    if (mode != FR_MODE_SCORES && c->cheb_n == 0) raise(FR_ERR_INVALID_ARG, "context has no Chebyshev degree");
    if (mode != FR_MODE_SCORES && L - 1 - c->cmp_depth < 0) raise(FR_ERR_LEVEL, "not enough levels for the threshold");
    if (mode != FR_MODE_SCORES && mode != FR_MODE_IDENTIFY && mode != FR_MODE_MEMBERSHIP)
        raise(FR_ERR_INVALID_ARG, "unknown mode");
    CU(cudaSetDevice(c->device));
    const int L1 = L + 1;
    int nout0, lo;
    match_shape(c, dbs[0], mode, &nout0, &lo);
    std::vector<long long> first;
    const long long tot = match_outputs(dbs, mode, first);
    const size_t ow = (size_t)ctw(c, lo + 1), iw = (size_t)ctw(c, L1);
    auto oblk = new_block(c, (size_t)tot * ow);
    if (c->prof && c->use_graphs) {
        // profiled replay: the match is captured with its region events as graph nodes and
        // replayed once, so the regions are timed back to back as in a graph replay (no host
        // launch gaps inside them)
        Tmp q(c, (size_t)B * iw);
        for (int b = 0; b < B; ++b) to_device(c, queries[b], q.p + (size_t)b * iw, L1, L);
        cudaEvent_t pa = nullptr, pb = nullptr;
        CU(cudaEventCreate(&pa));
        CU(cudaEventCreate(&pb));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        CU(cudaStreamBeginCapture(c->cur, cudaStreamCaptureModeThreadLocal));
        try {
            match_pipeline(c, dbs, q.p, mode, oblk->p);
        } catch (...) {
            if (cudaStreamEndCapture(c->cur, &graph) == cudaSuccess && graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            cudaEventDestroy(pa);
            cudaEventDestroy(pb);
            throw;
        }
        CU(cudaStreamEndCapture(c->cur, &graph));
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CU(ie);
        CU(cudaEventRecord(pa, c->cur));
        const cudaError_t le = cudaGraphLaunch(exec, c->cur);
        CU(cudaEventRecord(pb, c->cur));
        CU(cudaStreamSynchronize(c->cur));
        cudaGraphExecDestroy(exec);
        // a profiled graph is replayed once: hand the memory its allocations reserved back to
        // the device, so that repeated profiled matches do not accumulate graph memory
        cudaDeviceGraphMemTrim(c->device);
        CU(le);
        Region& whole = c->regions["match"];
        whole.pending.emplace_back(pa, pb);
        whole.launches++;
    } else if (c->prof || !c->use_graphs) {
        Tmp q(c, (size_t)B * iw);
        for (int b = 0; b < B; ++b) to_device(c, queries[b], q.p + (size_t)b * iw, L1, L);
        match_pipeline(c, dbs, q.p, mode, oblk->p);
    } else {
        std::lock_guard<std::mutex> lock(g_graph_mu);
        const auto key = std::make_tuple((const fr_ctx*)c, dbs, (int)mode);
        if (!g_graphs.count(key)) {
            // at most kMaxGraphs graphs per context (each holds the workspace of its batch):
            // drop the least used one first
            constexpr size_t kMaxGraphs = 16;
            size_t mine = 0;
            auto victim = g_graphs.end();
            for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it) {
                if (std::get<0>(it->first) != c) continue;
                ++mine;
                if (victim == g_graphs.end() || it->second.runs < victim->second.runs) victim = it;
            }
            if (mine >= kMaxGraphs && victim != g_graphs.end()) {
                CU(cudaStreamSynchronize(c->cur));
                if (victim->second.exec) cudaGraphExecDestroy(victim->second.exec);
                cudaFree(victim->second.in);
                cudaFree(victim->second.out);
                g_graphs.erase(victim);
            }
        }
        MatchGraph& mg = g_graphs[key];
        if (!mg.in) {
            CU(cudaMalloc(&mg.in, (size_t)B * iw * 8));
            CU(cudaMalloc(&mg.out, (size_t)tot * ow * 8));
        }
        for (int b = 0; b < B; ++b) to_device(c, queries[b], mg.in + (size_t)b * iw, L1, L);
        if (!mg.exec && mg.runs >= 1) {
            const uint64_t k0 = c->launches;
            cudaGraph_t graph;
            CU(cudaStreamBeginCapture(c->cur, cudaStreamCaptureModeThreadLocal));
            try {
                match_pipeline(c, dbs, mg.in, mode, mg.out);
            } catch (...) {
                graph = nullptr;
                if (cudaStreamEndCapture(c->cur, &graph) == cudaSuccess && graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                throw;
            }
            CU(cudaStreamEndCapture(c->cur, &graph));
            CU(cudaGraphInstantiate(&mg.exec, graph, 0));
            cudaGraphDestroy(graph);
            mg.kernels = c->launches - k0;
            c->launches = k0;
        }
        if (mg.exec) {
            CU(cudaGraphLaunch(mg.exec, c->cur));
            c->launches += mg.kernels;
        } else {
            match_pipeline(c, dbs, mg.in, mode, mg.out);
        }
        mg.runs++;
        copy_d2d(c, oblk->p, mg.out, (size_t)tot * ow);
    }
    fr_ct** arr = new fr_ct*[tot];
    for (long long i = 0; i < tot; ++i) arr[i] = new_dev_ct(c, oblk, oblk->p + (size_t)i * ow, lo, lo + 1);
    *out = arr;
    *n_out = (size_t)tot;
}

void check_match_args(fr_ctx* c, const fr_db* db, const fr_ct* q, fr_mode mode) {
    need_device(c);
    if (!db) raise(FR_ERR_INVALID_ARG, "null database");
    if (db->ctx != c) raise(FR_ERR_INVALID_ARG, "database belongs to another context");
    check_ct(c, q);
    if (q->level != c->R.nq - 1) raise(FR_ERR_LEVEL, "queries must be at the top level");
    if (mode != FR_MODE_SCORES && mode != FR_MODE_IDENTIFY && mode != FR_MODE_MEMBERSHIP)
        raise(FR_ERR_INVALID_ARG, "unknown mode");
    if (mode != FR_MODE_SCORES && c->cheb_n == 0) raise(FR_ERR_INVALID_ARG, "context has no Chebyshev degree");
    if (mode != FR_MODE_SCORES && c->work_level - 1 - c->cmp_depth < 0) raise(FR_ERR_LEVEL, "not enough levels for the threshold");
}

// ---------------------------------------------------------------------------
// Serving loop (continuous batching). fr_match_submit queues a request. A worker
// thread forms a batch from the oldest request's (database, mode) class, admits it
// when a slot (a stream pair of its own) is free and the batch's workspace fits the
// HBM left by the batches in flight, enqueues it through match_pipeline on the slot's
// streams and goes on admitting; slots retire as their work completes (a host callback
// after the batch's last operation wakes the worker), so batches overlap on the device
// while new requests keep arriving. fr_match_poll waits for a ticket's outputs.
// ---------------------------------------------------------------------------
using ServeClock = std::chrono::steady_clock;

struct ServeReq {
    uint64_t ticket = 0;
    ServeClock::time_point t_submit;
    const fr_db* db = nullptr;
    fr_mode mode = FR_MODE_SCORES;
    fr_ct q;  // private copy: host words of the working-level limbs, or the shared device block
};

struct ServeResult {
    double latency_ms = 0;  // submit -> end of the batch's device work
    fr_status st = FR_OK;
    std::string err;
    std::shared_ptr<DevBlock> blk;
    size_t first = 0;  // word offset of the request's first output
    int nout = 0, lo = 0;
    size_t ow = 0;
};

struct ServeSlot {
    cudaStream_t s = nullptr, side = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    bool finished = false;  // set by the host callback enqueued after the batch
    ServeClock::time_point t_finish;
    const fr_db* db = nullptr;
    std::vector<uint64_t> tickets;
    std::vector<ServeClock::time_point> t_submit;
    std::shared_ptr<DevBlock> out;
    int nout = 0, lo = 0;
    size_t ow = 0;
    uint64_t reserved = 0;
    std::string err;
};

struct SlotCb {
    Server* S;
    int k;
};

}  // namespace

struct Server {
    fr_ctx* c = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;       // worker: new request, finished slot, stop
    std::condition_variable cv_done;  // pollers
    std::deque<ServeReq> pending;
    std::map<uint64_t, ServeResult> done;
    std::set<uint64_t> inflight;
    std::vector<ServeSlot> slots;
    std::vector<SlotCb> cbs;
    uint32_t max_batch = 8;
    uint64_t avail = 0, reserved = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    uint64_t n_done = 0, n_batches = 0, max_busy = 0;
};

namespace {

// Upper bound of the device workspace of one batch: base + B * per_query bytes.
void match_workspace(const fr_ctx* c, const fr_db* db, fr_mode mode, uint64_t* base, uint64_t* per_query) {
    const double N = c->R.N;
    const int L = c->work_level, L1 = L + 1;
    const double n1 = c->n1, ell = c->ell, n2 = std::ceil(ell / n1), G = (double)db->G;
    const double beta = c->R.digits_at(L), npos = L1 + c->R.np;
    const double cw1 = 2.0 * L1 * N, cw = 2.0 * L * N;
    int nout, lo;
    match_shape(c, db, mode, &nout, &lo);
    double per = cw1 + nout * 2.0 * (lo + 1) * N + G * cw;
    const double bwq = db->schedule != 1 && c->hoist_babies ? 2.0 * npos * N : cw1;  // one baby / giant-step sum
    if (db->schedule != 1) per += (n1 + n2) * bwq + 2.0 * n2 * cw;
    if (mode != FR_MODE_SCORES) per += G * 54.0 * cw;  // threshold: powers, leaves, tree temporaries
    // key-switch scratch: ModUp of 16 inputs, 32 accumulators, 32 tensor products
    double b = 16.0 * (2.0 * L1 + beta * npos) * N + 32.0 * 2.0 * npos * N + 32.0 * 3.0 * L1 * N;
    if (db->schedule == 1) b += ell * cw1 + G * cw1;
    if (db->tier == 4) per += 3.0 * n2 * L1 * N;  // unrelinearised products of the giant steps
    if (db->tier != 1 && db->tier != 4) b += (db->schedule == 1 ? std::min(G, 8.0) : 1.0) * ell * db->nl * N;
    *base = (uint64_t)(b * 8.0 * 1.25);
    *per_query = (uint64_t)(per * 8.0 * 1.25);
}

void CUDART_CB slot_finished(void* p) {
    SlotCb* cb = static_cast<SlotCb*>(p);
    {
        std::lock_guard<std::mutex> lk(cb->S->mu);
        cb->S->slots[cb->k].finished = true;
        cb->S->slots[cb->k].t_finish = ServeClock::now();
    }
    cb->S->cv.notify_all();
}

// Move finished slots' outputs to the done map. Called with S->mu held.
void serve_retire(Server* S) {
    bool any = false;
    for (auto& sl : S->slots) {
        if (!sl.busy || !sl.finished) continue;
        const cudaError_t e = sl.err.empty() ? cudaEventQuery(sl.ev) : cudaSuccess;
        for (size_t b = 0; b < sl.tickets.size(); ++b) {
            ServeResult r;
            r.latency_ms = std::chrono::duration<double, std::milli>(sl.t_finish - sl.t_submit[b]).count();
            if (!sl.err.empty()) {
                r.st = FR_ERR_CUDA;
                r.err = sl.err;
            } else if (e != cudaSuccess) {
                r.st = FR_ERR_CUDA;
                r.err = std::string("batch failed on the device: ") + cudaGetErrorString(e);
            } else {
                r.blk = sl.out;
                r.first = b * (size_t)sl.nout * sl.ow;
                r.nout = sl.nout;
                r.lo = sl.lo;
                r.ow = sl.ow;
            }
            S->done[sl.tickets[b]] = std::move(r);
            S->inflight.erase(sl.tickets[b]);
        }
        S->n_done += sl.tickets.size();
        S->n_batches++;
        S->reserved -= sl.reserved;
        sl.busy = false;
        sl.finished = false;
        sl.tickets.clear();
        sl.db = nullptr;
        sl.err.clear();
        sl.out.reset();
        any = true;
    }
    if (any) S->cv_done.notify_all();
}

// Admit one batch if a slot is free and memory allows. Called with lk held; releases
// it while the batch is enqueued. Returns true when a batch was launched.
bool serve_admit(Server* S, std::unique_lock<std::mutex>& lk) {
    fr_ctx* c = S->c;
    int k = -1;
    for (size_t i = 0; i < S->slots.size(); ++i)
        if (!S->slots[i].busy) { k = (int)i; break; }
    if (k < 0 || S->pending.empty()) return false;
    // classes in arrival order: requests with the oldest request's (database, mode) are class 0
    const size_t n = S->pending.size();
    std::vector<uint32_t> cls(n), idx(std::max<uint32_t>(S->max_batch, 1));
    const fr_db* db = S->pending[0].db;
    const fr_mode mode = S->pending[0].mode;
    for (size_t i = 0; i < n; ++i) cls[i] = (S->pending[i].db == db && S->pending[i].mode == mode) ? 0u : 1u;
    uint64_t ws_base, ws_q;
    match_workspace(c, db, mode, &ws_base, &ws_q);
    const uint64_t free_now = S->avail > S->reserved ? S->avail - S->reserved : 0;
    int B = frh::plan_batch(cls.data(), n, S->max_batch, free_now, ws_base, ws_q, idx.data());
    if (B == 0) {
        if (S->reserved > 0) return false;  // wait for batches in flight to release memory
        B = 1;                              // nothing in flight: run the oldest request alone
        idx[0] = 0;
    }
    std::vector<ServeReq> batch;
    {
        std::vector<bool> take(n, false);
        for (int b = 0; b < B; ++b) take[idx[b]] = true;
        std::deque<ServeReq> rest;
        for (size_t i = 0; i < n; ++i) {
            if (take[i]) batch.push_back(std::move(S->pending[i]));
            else rest.push_back(std::move(S->pending[i]));
        }
        S->pending.swap(rest);
    }
    ServeSlot& sl = S->slots[k];
    sl.busy = true;
    sl.finished = false;
    sl.db = db;
    sl.tickets.clear();
    sl.t_submit.clear();
    for (auto& r : batch) {
        sl.tickets.push_back(r.ticket);
        sl.t_submit.push_back(r.t_submit);
        S->inflight.insert(r.ticket);
    }
    sl.reserved = ws_base + (uint64_t)B * ws_q;
    S->reserved += sl.reserved;
    uint64_t busy = 0;
    for (auto& x : S->slots) busy += x.busy;
    S->max_busy = std::max(S->max_busy, busy);
    lk.unlock();
    std::string err;
    try {
        std::lock_guard<std::recursive_mutex> cl(c->mu);
        struct Swap {
            fr_ctx* c;
            cudaStream_t cur, side;
            ~Swap() { c->cur = cur; c->side = side; }
        } swap{c, c->cur, c->side};
        c->cur = sl.s;
        c->side = sl.side;
        const int L = c->work_level, L1 = L + 1;
        int nout, lo;
        match_shape(c, db, mode, &nout, &lo);
        const size_t ow = (size_t)ctw(c, lo + 1), iw = (size_t)ctw(c, L1);
        auto oblk = new_block(c, (size_t)B * nout * ow);
        {
            Tmp q(c, (size_t)B * iw);
            for (int b = 0; b < B; ++b) to_device(c, &batch[b].q, q.p + (size_t)b * iw, L1, L);
            match_pipeline(c, std::vector<const fr_db*>(B, db), q.p, mode, oblk->p);
        }
        CU(cudaEventRecord(sl.ev, sl.s));
        sl.out = oblk;
        sl.nout = nout;
        sl.lo = lo;
        sl.ow = ow;
        CU(cudaLaunchHostFunc(sl.s, slot_finished, &S->cbs[k]));
    } catch (const FrError& e) {
        err = e.msg.empty() ? "batch failed" : e.msg;
    } catch (const std::exception& e) {
        err = e.what();
    }
    lk.lock();
    if (!err.empty()) {
        // nothing more was enqueued after the failure: retire the slot with the error
        sl.err = err;
        sl.finished = true;
        sl.t_finish = ServeClock::now();
        sl.out.reset();
    }
    return true;
}

void serve_loop(Server* S) {
    cudaSetDevice(S->c->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        serve_retire(S);
        bool busy = false;
        for (auto& sl : S->slots) busy = busy || sl.busy;
        if (S->stop && S->pending.empty() && !busy) break;
        bool launched = false;
        while (!S->pending.empty() && serve_admit(S, lk)) {
            launched = true;
            serve_retire(S);
        }
        if (launched) continue;
        S->cv.wait(lk);
    }
}

void serve_start(fr_ctx* c, uint32_t max_batch, uint32_t nslots, uint64_t budget) {
    if (c->server) raise(FR_ERR_INVALID_ARG, "the serving loop is already running");
    if (max_batch < 1 || max_batch > 64) raise(FR_ERR_INVALID_ARG, "max_batch must be 1..64");
    if (nslots < 1 || nslots > 8) raise(FR_ERR_INVALID_ARG, "slots must be 1..8");
    CU(cudaSetDevice(c->device));
    std::unique_ptr<Server> S(new Server());
    S->c = c;
    S->max_batch = max_batch;
    if (budget) {
        S->avail = budget;
    } else {
        size_t free_b = 0, total_b = 0;
        CU(cudaMemGetInfo(&free_b, &total_b));
        const size_t margin = (size_t)4 << 30;
        S->avail = free_b > margin ? free_b - margin : 0;
    }
    S->slots.resize(nslots);
    for (uint32_t k = 0; k < nslots; ++k) {
        CU(cudaStreamCreateWithFlags(&S->slots[k].s, cudaStreamNonBlocking));
        CU(cudaStreamCreateWithFlags(&S->slots[k].side, cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&S->slots[k].ev, cudaEventDisableTiming));
        S->cbs.push_back(SlotCb{S.get(), (int)k});
    }
    Server* sp = S.get();
    S->th = std::thread([sp] { serve_loop(sp); });
    c->server = S.release();
}

void serve_shutdown(fr_ctx* c) {
    Server* S = c->server;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    for (auto& sl : S->slots) {
        cudaStreamSynchronize(sl.s);
        cudaStreamSynchronize(sl.side);
    }
    S->done.clear();
    for (auto& sl : S->slots) {
        cudaEventDestroy(sl.ev);
        cudaStreamDestroy(sl.s);
        cudaStreamDestroy(sl.side);
    }
    c->server = nullptr;
    delete S;
}

void serve_drain_db(fr_ctx* c, const fr_db* db) {
    Server* S = c ? c->server : nullptr;
    if (!S) return;
    std::unique_lock<std::mutex> lk(S->mu);
    auto uses = [&] {
        for (auto& r : S->pending)
            if (r.db == db) return true;
        for (auto& sl : S->slots)
            if (sl.busy && sl.db == db) return true;
        return false;
    };
    S->cv_done.wait(lk, [&] { return !uses(); });
}

}  // namespace

extern "C" {

fr_status fr_serve_start(fr_ctx* c, const fr_serve_params* p) {
    return guard([&] {
        need_device(c);
        serve_start(c, p ? p->max_batch : 8, p ? p->slots : 2, p ? p->hbm_budget_bytes : 0);
    });
}

fr_status fr_serve_stop(fr_ctx* c) {
    return guard([&] {
        need_device(c);
        serve_shutdown(c);
    });
}

fr_status fr_match_submit(fr_ctx* c, const fr_db* db, const fr_ct* query, fr_mode mode, uint64_t* ticket) {
    return guard([&] {
        if (!ticket) raise(FR_ERR_INVALID_ARG, "null ticket pointer");
        check_match_args(c, db, query, mode);
        if (!c->server) serve_start(c, 8, 2, 0);
        ServeReq r;
        r.db = db;
        r.mode = mode;
        const int L = c->work_level, N = c->R.N;
        r.q.ctx = c;
        r.q.scale = query->scale;
        if (query->on_dev) {
            r.q = *query;
        } else {
            // keep only the limbs the match uses (the query is dropped to the working level)
            r.q.level = L;
            r.q.cap = L + 1;
            r.q.on_dev = false;
            r.q.host.resize((size_t)2 * (L + 1) * N);
            const size_t src_l = (size_t)query->level + 1;
            for (int t = 0; t < 2; ++t)
                std::memcpy(r.q.host.data() + (size_t)t * (L + 1) * N, query->host.data() + (size_t)t * src_l * N,
                            (size_t)(L + 1) * N * 8);
        }
        Server* S = c->server;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            r.ticket = S->next_ticket++;
            r.t_submit = ServeClock::now();
            *ticket = r.ticket;
            S->pending.push_back(std::move(r));
        }
        S->cv.notify_all();
    });
}

fr_status fr_match_poll(fr_ctx* c, uint64_t ticket, int block_ms, fr_ct*** out, size_t* n_out, double* latency_ms) {
    return guard([&] {
        need_device(c);
        if (!out || !n_out) raise(FR_ERR_INVALID_ARG, "null argument");
        Server* S = c->server;
        if (!S) raise(FR_ERR_INVALID_ARG, "no serving loop on this context");
        ServeResult r;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            auto known = [&] {
                if (S->done.count(ticket) || S->inflight.count(ticket)) return true;
                for (auto& q : S->pending)
                    if (q.ticket == ticket) return true;
                return false;
            };
            if (!known()) raise(FR_ERR_INVALID_ARG, "unknown ticket");
            auto ready = [&] { return S->done.count(ticket) > 0; };
            if (!ready()) {
                if (block_ms < 0) S->cv_done.wait(lk, ready);
                else if (block_ms > 0) S->cv_done.wait_for(lk, std::chrono::milliseconds(block_ms), ready);
            }
            if (!ready()) raise(FR_ERR_TIMEOUT, "request not finished");
            r = std::move(S->done[ticket]);
            S->done.erase(ticket);
        }
        if (latency_ms) *latency_ms = r.latency_ms;
        if (r.st != FR_OK) raise(r.st, r.err);
        fr_ct** arr = new fr_ct*[r.nout];
        for (int i = 0; i < r.nout; ++i) arr[i] = new_dev_ct(c, r.blk, r.blk->p + r.first + (size_t)i * r.ow, r.lo, r.lo + 1);
        *out = arr;
        *n_out = (size_t)r.nout;
    });
}

fr_status fr_serve_stats(fr_ctx* c, uint64_t* completed, uint64_t* batches, uint64_t* pending,
                         uint64_t* max_concurrent) {
    return guard([&] {
        need_device(c);
        Server* S = c->server;
        uint64_t a = 0, b = 0, p = 0, m = 0;
        if (S) {
            std::lock_guard<std::mutex> lk(S->mu);
            a = S->n_done;
            b = S->n_batches;
            p = S->pending.size() + S->inflight.size();
            m = S->max_busy;
        }
        if (completed) *completed = a;
        if (batches) *batches = b;
        if (pending) *pending = p;
        if (max_concurrent) *max_concurrent = m;
    });
}

fr_status fr_serve_plan(const uint32_t* classes, size_t n, uint32_t max_batch, uint64_t avail_bytes,
                        uint64_t ws_base, uint64_t ws_per_query, uint32_t* chosen, size_t* n_chosen) {
    return guard([&] {
        if ((n && !classes) || !chosen || !n_chosen) raise(FR_ERR_INVALID_ARG, "null argument");
        std::vector<uint32_t> idx(std::max<uint32_t>(max_batch, 1));
        const int B = frh::plan_batch(classes, n, max_batch, avail_bytes, ws_base, ws_per_query, idx.data());
        for (int b = 0; b < B; ++b) chosen[b] = idx[b];
        *n_chosen = (size_t)B;
    });
}

}  // extern "C"

extern "C" {

fr_status fr_match(fr_ctx* c, const fr_db* db, const fr_ct* query, fr_mode mode, fr_ct*** out, size_t* n_out) {
    return guard([&] {
        if (!c) raise(FR_ERR_INVALID_ARG, "null context");
        const fr_ct* qs[1] = {query};
        match_queries(c, std::vector<const fr_db*>(1, db), qs, mode, out, n_out);
    });
}

fr_status fr_match_batch(fr_ctx* c, const fr_db* db, const fr_ct* const* queries, size_t n_queries, fr_mode mode,
                         fr_ct*** out, size_t* n_out) {
    return guard([&] {
        if (!c) raise(FR_ERR_INVALID_ARG, "null context");
        if (n_queries > 64) raise(FR_ERR_INVALID_ARG, "at most 64 queries per batch");
        match_queries(c, std::vector<const fr_db*>(n_queries, db), queries, mode, out, n_out);
    });
}

fr_status fr_match_multi(fr_ctx* c, const fr_db* const* dbs, const fr_ct* const* queries, size_t n_queries,
                         fr_mode mode, fr_ct*** out, size_t* n_out) {
    return guard([&] {
        if (!c) raise(FR_ERR_INVALID_ARG, "null context");
        if (!dbs) raise(FR_ERR_INVALID_ARG, "null argument");
        if (n_queries > 64) raise(FR_ERR_INVALID_ARG, "at most 64 queries per batch");
        match_queries(c, std::vector<const fr_db*>(dbs, dbs + n_queries), queries, mode, out, n_out);
    });
}

fr_status fr_sync(fr_ctx* c) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        CU(cudaStreamSynchronize(c->cur));
    });
}

fr_status fr_profile(fr_ctx* c, int enable) {
    return guard([&] {
        if (!c) raise(FR_ERR_INVALID_ARG, "null argument");
        CU(cudaStreamSynchronize(c->cur));
        for (auto& r : c->regions) {
            for (auto& e : r.second.pending) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
            r.second.pending.clear();
            r.second.ms = 0;
            r.second.launches = 0;
            r.second.bytes = 0;
        }
        c->prof = enable != 0;
    });
}

fr_status fr_profile_only(fr_ctx* c, const char* prefix) {
    return guard([&] {
        if (!c) raise(FR_ERR_INVALID_ARG, "null argument");
        c->prof_only = prefix ? prefix : "";
    });
}

fr_status fr_profile_read(fr_ctx* c, const char* region, double* ms, uint64_t* launches, uint64_t* bytes) {
    return guard([&] {
        if (!c || !region) raise(FR_ERR_INVALID_ARG, "null argument");
        CU(cudaStreamSynchronize(c->cur));
        Region& r = c->regions[region];
        for (auto& e : r.pending) {
            float t = 0;
            CU(cudaEventElapsedTime(&t, e.first, e.second));
            r.ms += t;
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
        r.pending.clear();
        if (ms) *ms = r.ms;
        if (launches) *launches = r.launches;
        if (bytes) *bytes = r.bytes;
    });
}

uint64_t fr_launch_count(const fr_ctx* c) { return c ? c->launches : 0; }

fr_status fr_ctx_primes(const fr_ctx* c, uint64_t* out, size_t cap, size_t* n) {
    if (!c || !n) return FR_ERR_INVALID_ARG;
    *n = c->R.primes.size();
    for (size_t i = 0; i < c->R.primes.size() && i < cap && out; ++i) out[i] = c->R.primes[i];
    return FR_OK;
}

fr_status fr_ctx_info(const fr_ctx* c, uint32_t* n_slots, uint32_t* top_level, uint32_t* n_digits,
                      uint64_t* resident_bytes) {
    if (!c) return FR_ERR_INVALID_ARG;
    if (n_slots) *n_slots = (uint32_t)c->R.N / 2;
    if (top_level) *top_level = (uint32_t)c->R.nq - 1;
    if (n_digits) *n_digits = (uint32_t)c->R.ndig;
    if (resident_bytes) *resident_bytes = c->resident;
    return FR_OK;
}

uint32_t fr_work_level(const fr_ctx* c) { return c ? (uint32_t)c->work_level : 0; }

fr_status fr_ntt_tuning(const fr_ctx* c, uint32_t* shapes, double* us) {
    return guard([&] {
        need_device(c);
        for (int b = 0; b < FR_NTT_BUCKETS; ++b) {
            if (shapes) shapes[b] = c->rd.ntt_shape[b];
            for (int sh = 0; sh < FR_NTT_SHAPES && us; ++sh)
                us[b * FR_NTT_SHAPES + sh] = c->ntt_tune_us[b * FR_NTT_SHAPES + sh];
        }
    });
}

fr_status fr_ntt_set_shapes(fr_ctx* c, const uint32_t* shapes) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        if (!shapes) raise(FR_ERR_INVALID_ARG, "null argument");
        for (int b = 0; b < FR_NTT_BUCKETS; ++b)
            if (shapes[b] >= FR_NTT_SHAPES) raise(FR_ERR_INVALID_ARG, "NTT tile shape must be 0..5");
        for (int b = 0; b < FR_NTT_BUCKETS; ++b) c->rd.ntt_shape[b] = (unsigned char)shapes[b];
        drop_graphs(c, nullptr);  // captured graphs hold the previous launch shapes
    });
}

fr_status fr_set_db_tier(fr_ctx* c, uint32_t tier) {
    return guard([&] {
        need_device(c);
        if (tier > 3) raise(FR_ERR_INVALID_ARG, "db_tier must be 0, 1, 2 or 3");
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        c->db_tier = tier;
    });
}

fr_status fr_use_graphs(fr_ctx* c, int on) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        c->use_graphs = on != 0;
    });
}

fr_status fr_inject_alloc_failure(fr_ctx* c, int64_t after) {
    return guard([&] {
        if (!c) raise(FR_ERR_INVALID_ARG, "null context");
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        c->fail_alloc_after = after < 0 ? -1 : (long long)after;
    });
}

fr_status fr_ntt_time(fr_ctx* c, uint32_t npolys, uint32_t level, uint32_t reps, double* us_fwd, double* us_inv) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        if (npolys == 0 || reps == 0 || !us_fwd || !us_inv) raise(FR_ERR_INVALID_ARG, "bad argument");
        if ((int)level >= c->R.nq) raise(FR_ERR_LEVEL, "level out of range");
        CU(cudaSetDevice(c->device));
        const size_t words = (size_t)npolys * c->R.N;
        Tmp buf(c, words);
        CU(cudaMemsetAsync(buf.p, 0, words * 8, c->cur));
        const PrimeMap pm = pm_level((int)level);
        const PolyBatch pb{buf.p, (long long)(level + 1) * c->R.N, (int)level + 1, (int)npolys, pm};
        cudaEvent_t a, b;
        CU(cudaEventCreate(&a));
        CU(cudaEventCreate(&b));
        double best[2] = {1e30, 1e30};
        for (uint32_t r = 0; r <= reps; ++r) {  // the first round warms up
            for (int inv = 0; inv < 2; ++inv) {
                cudaEventRecord(a, c->cur);
                launch_ntt(c->rd, pb, inv != 0, c->cur);
                cudaEventRecord(b, c->cur);
                cudaEventSynchronize(b);
                float ms = 0;
                cudaEventElapsedTime(&ms, a, b);
                if (r > 0) best[inv] = std::min(best[inv], 1000.0 * ms);
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        CU(cudaGetLastError());
        *us_fwd = best[0];
        *us_inv = best[1];
    });
}

fr_status fr_butterfly_peak(int device, double* butterflies_per_s) {
    return guard([&] {
        if (!butterflies_per_s) raise(FR_ERR_INVALID_ARG, "null argument");
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
            raise(FR_ERR_CUDA, "no such CUDA device");
        CU(cudaSetDevice(device));
        *butterflies_per_s = measure_butterfly_peak(device);
        CU(cudaGetLastError());
    });
}

fr_status fr_fp64_peak(int device, double* flops_per_s) {
    return guard([&] {
        if (!flops_per_s) raise(FR_ERR_INVALID_ARG, "null argument");
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
            raise(FR_ERR_CUDA, "no such CUDA device");
        CU(cudaSetDevice(device));
        *flops_per_s = measure_fp64_peak(device);
        CU(cudaGetLastError());
    });
}

fr_status fr_cheb_coeffs(uint32_t n, double tau, double* out) { return fr_cheb_coeffs_lo(n, tau, 0.0, out); }

fr_status fr_cheb_coeffs_lo(uint32_t n, double tau, double low, double* out) {
    if (!out) return FR_ERR_INVALID_ARG;
    std::vector<double> c;
    frh::cheb_coeffs((int)n, tau, c, low);
    std::copy(c.begin(), c.end(), out);
    return FR_OK;
}

}  // extern "C"

// ===========================================================================
// Rotation that allocates nothing.
//
// Some callers cannot allocate device memory while they run: code that is
// being captured into a CUDA graph with a fixed memory plan, an inference
// server whose request path must not touch the allocator (to avoid pool
// growth and its synchronisation), or a host that has handed all free HBM to
// another owner. fr_rotate_noalloc serves them: the caller passes input and
// output buffers, and every temporary of the key switch lives in the fixed
// device array below, compiled into the library. That array is
// FR_NOALLOC_SCRATCH_WORDS words (64 MiB) and every GPU that loads this part
// of the library keeps it until the process exits.
// ===========================================================================
#define FR_NOALLOC_SCRATCH_WORDS (8ull << 20)
static __device__ __align__(256) u64 g_noalloc_scratch[FR_NOALLOC_SCRATCH_WORDS];

namespace {
// Device address of the scratch array on `device` (looked up once per device,
// with that device current). In host code the array's name is only a
// host-side stand-in, so kernels must be given this address instead.
constexpr int kMaxDevices = 64;  // device ordinals the address cache covers
u64* noalloc_scratch(int device) {
    static std::mutex mu;
    static u64* addr[kMaxDevices] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (device < 0 || device >= kMaxDevices) raise(FR_ERR_INVALID_ARG, "device ordinal out of range");
    if (!addr[device]) {
        void* p = nullptr;
        CU(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        addr[device] = (u64*)p;
    }
    return addr[device];
}
}  // namespace

extern "C" fr_status fr_rotate_noalloc(fr_ctx* c, const uint64_t* d_in, uint32_t level, int32_t k,
                                       uint64_t* d_out) {
    return guard([&] {
        need_device(c);
        std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
        if (!d_in || !d_out) raise(FR_ERR_INVALID_ARG, "null buffer");
        if ((int)level >= c->R.nq) raise(FR_ERR_LEVEL, "level out of range");
        // every argument is checked before anything is enqueued, so a refused call leaves
        // nothing on the stream (or in a graph being captured)
        if ((int)level > c->key_level) raise(FR_ERR_LEVEL, "the loaded keys stop at the context's working level");
        CU(cudaSetDevice(c->device));
        const int N = c->R.N, l = (int)level, np = c->R.np, nq = c->R.nq;
        const size_t L1N = (size_t)(l + 1) * N;
        const u64 g = frh::galois_of_rotation(c->R, k);
        if (g == 1) {
            CU(cudaMemcpyAsync(d_out, d_in, 2 * L1N * 8, cudaMemcpyDeviceToDevice, c->cur));
            return;
        }
        const u64* key = rot_key(c, g);
        const int npos = l + 1 + np, beta = c->R.digits_at(l);
        const size_t need = 5 * L1N + (size_t)(beta + 2) * npos * N;
        if (need > FR_NOALLOC_SCRATCH_WORDS)
            raise(FR_ERR_INVALID_ARG, "fr_rotate_noalloc: needs " + std::to_string(need) +
                                          " scratch words at this level, the fixed array holds " +
                                          std::to_string(FR_NOALLOC_SCRATCH_WORDS));
        u64* sc = noalloc_scratch(c->device);
        u64* e = sc;                     // [2][l+1][N] input, evaluation form
        u64* a = e + 2 * L1N;            // [l+1][N] c1, coefficient form
        u64* ext = a + L1N;              // [beta][npos][N]
        u64* acc = ext + (size_t)beta * npos * N;  // [2][npos][N]
        u64* conv = acc + (size_t)2 * npos * N;    // [2][l+1][N]
        cudaStream_t st = c->cur;
        CU(cudaMemcpyAsync(e, d_in, 2 * L1N * 8, cudaMemcpyDeviceToDevice, st));
        CU(cudaMemcpyAsync(a, d_in + L1N, L1N * 8, cudaMemcpyDeviceToDevice, st));
        const PrimeMap pl = pm_level(l);
        launch_ntt(c->rd, PolyBatch{e, (long long)N, 2 * (l + 1), 2 * (l + 1), pl}, false, st);
        launch_modup(a, 0, e + L1N, 0, ext, c->d_modup[l], beta, npos, N, 1, st);
        launch_ntt(c->rd, PolyBatch{ext, (long long)beta * npos * N, 1, c->modup_ntt_n[l], PrimeMap{},
                                    c->d_modup_ntt[l], c->modup_ntt_n[l]},
                   false, st);
        IPJobs ij;
        ij.j[0] = IPJob{ext, key, acc, (u32)g, 0};
        ij.gkey[0] = key;
        ij.gstart[0] = 0;
        ij.gstart[1] = 1;
        ij.ngroups = 1;
        launch_ip(ij, beta, npos, l, c->key_level + 1, c->key_limbs, c->d_primes, pm_ext(c, l), c->R.logN, st);
        PrimeMap pmP{};
        pmP.period = np;
        for (int j = 0; j < np; ++j) pmP.idx[j] = (unsigned char)(nq + j);
        launch_ntt(c->rd, PolyBatch{acc + L1N, (long long)npos * N, np, 2 * np, pmP}, true, st);
        launch_p2q(acc, 2ll * npos * N, npos, l, conv, c->d_p2q, N, 1, st);
        launch_ntt(c->rd, PolyBatch{conv, (long long)L1N, l + 1, 2 * (l + 1), pl}, false, st);
        MDJobs md;
        md.j[0] = MDJob{acc, conv, e, d_out, l + 1, l + 1, 1, (u32)g};
        launch_moddown_combine(md, 1, npos, l, c->d_pinv, c->d_pinv_s, c->d_primes, c->R.logN, st);
        launch_ntt(c->rd, PolyBatch{d_out, (long long)N, 2 * (l + 1), 2 * (l + 1), pl}, true, st);
        c->launches += 13;
        CU(cudaGetLastError());
    });
}
