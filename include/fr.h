/*
 * fr.h -- C ABI of the GB300 encrypted 1:N face-matching library.
 *
 * The library computes, on one GPU, the server side of the encrypted
 * similarity search of "Lightweight, Practical Encrypted Face Recognition with
 * GPU Support" (arXiv 2604.00546): a CKKS plaintext-template-matrix times
 * encrypted-query product by BSGS with hoisted baby steps and pre-rotated
 * diagonals (Section "BSGS with pre-rotated diagonals on GPU", Eq.
 * eq:prerotation, Algorithms 5 and 6), the Chebyshev threshold of Eq.
 * eq:cheb-sign (Paterson-Stockmeyer paragraph) and the membership slot sum
 * (Algorithm 5, aggregation step). The client side (key generation,
 * encryption, decryption; Fig. "HyDia protocol", Section "HyDia") runs on the
 * host.
 *
 * Conventions
 *  - Every call returns fr_status. On error the out-pointers are untouched and
 *    fr_last_error() (thread-local) describes the failure.
 *  - Inputs are copied; the caller keeps ownership. Outputs are library-owned
 *    handles released with the matching fr_free_* call.
 *  - A ciphertext in the exported format is coefficient form, limb-major
 *    uint64 [2][level+1][N], each word in [0, q_i), component 0 first; it
 *    decrypts as c0 + c1 * s.
 *  - Slots: n = N/2 real slots; slot j is the evaluation at zeta^(5^j mod 2N).
 *    A rotation by k moves slot j+k to slot j (left rotation).
 *  - Device work runs on the context stream (fr_params.cuda_stream, or a
 *    stream the context creates). Calls that return device handles enqueue
 *    work and return; calls that read results (fr_ct_export, fr_decrypt,
 *    fr_sync) wait for the stream.
 *  - There is no CPU fallback: without a usable CUDA device fr_setup fails
 *    with FR_ERR_CUDA.
 */
#ifndef FR_H
#define FR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fr_ctx fr_ctx;
typedef struct fr_keys fr_keys;
typedef struct fr_db fr_db;
typedef struct fr_ct fr_ct;

typedef enum {
    FR_OK = 0,
    FR_ERR_INVALID_ARG = 1,
    FR_ERR_HBM_BUDGET = 2,   /* resident + working set would exceed fr_params.hbm_budget_bytes */
    FR_ERR_CUDA = 3,         /* CUDA runtime error (no device, launch failure, out of memory) */
    FR_ERR_TIMEOUT = 4,      /* a bounded wait ran out */
    FR_ERR_LEVEL = 5,        /* ciphertext level too low / mismatched for the operation */
    FR_ERR_FORMAT = 6,       /* malformed ciphertext words (a residue >= q_i) */
    FR_ERR_INTERNAL = 7,
    FR_ERR_UNSUPPORTED = 8   /* valid but unsupported request (e.g. a Chebyshev degree with d1 != 2) */
} fr_status;

typedef enum {
    FR_MODE_SCORES = 0,      /* G ciphertexts of encrypted cosine scores (level L-1) */
    FR_MODE_IDENTIFY = 1,    /* G ciphertexts of p(score), p = Chebyshev step (Algorithm 6) */
    FR_MODE_MEMBERSHIP = 2   /* 1 ciphertext: sum over all slots of p(score) (Algorithm 5) */
} fr_mode;

/* Rotation-index sets for fr_rotation_set (paper: client-side key counts,
 * Section "Complexity analysis and memory consumption"; GPU complexity table). */
typedef enum {
    FR_KEYS_ONDEMAND = 0,    /* this library: baby {1..n1-1}, giant {j n1}, + powers of two if membership */
    FR_KEYS_CPU_BSGS = 1,    /* BSGS-Diagonal on CPU: baby + giant */
    FR_KEYS_HYDIA_DG = 2,    /* HyDia diagonal method: 1..ell-1 and EvalSum powers of two */
    FR_KEYS_TBS_ONLINE = 3,  /* server pre-rotation, keys resident online: giant + powers of two */
    FR_KEYS_TBS_TOTAL = 4,   /* server pre-rotation, all client keys: baby + giant + negative giant + powers */
    FR_KEYS_TBE_TOTAL = 5    /* enroller pre-rotation: baby + giant + powers */
} fr_keyset;

typedef struct {
    uint32_t log_n;            /* ring degree N = 2^log_n, 10 <= log_n <= 16 */
    uint32_t n_q;              /* number of ciphertext primes (top level L = n_q - 1) */
    const uint32_t* q_bits;    /* bit size of each Q prime, q_0 first (primes = 1 mod 2N, largest first) */
    uint32_t n_p;              /* number of special primes P */
    const uint32_t* p_bits;
    uint32_t dnum;             /* key-switching digits (capped at n_q); remainder limbs go to the last digits */
    uint32_t scale_bits;       /* Delta = 2^scale_bits */
    uint32_t ell;              /* template dimension (divides N/2) */
    uint32_t n1;               /* BSGS baby steps; n2 = ceil(ell / n1) */
    uint32_t schedule;         /* BSGS schedule: 0 on demand (Algorithms 5 and 6, diagonals pre-rotated per
                                  giant step, Eq. eq:prerotation); 1 the rotated-query table of Algorithm 1
                                  (all ell rotations of the query, plain diagonals); 2 auto: the table when
                                  ell - n1 < G (n2 - 1) and it fits in HBM. Fixed per database at fr_load_db. */
    uint32_t cheb_degree;      /* Chebyshev degree n of the threshold (PS split must give d1 = 2) */
    double threshold;          /* tau in step(x - tau) */
    uint64_t hbm_budget_bytes; /* 0: no budget beyond the device */
    int device;                /* CUDA device ordinal; -1: client-only context (host key generation,
                                  encryption, decryption; device calls fail with FR_ERR_CUDA) */
    void* cuda_stream;         /* optional cudaStream_t to run on (not owned); NULL: the context creates one */
    uint32_t db_tier;          /* template storage (plaintext diagonal tiers): 0 auto (tier 1 when the
                                  diagonals fit the budget / free HBM, else tier 3 when its coefficients
                                  fit, else tier 2); 1 (A) the pre-rotated diagonals are encoded once and
                                  kept in HBM in evaluation form at the working level; 3 (B) their rounded
                                  integer coefficients are kept (8 B per coefficient, 1/(level+1) of tier
                                  1) and each query forms the residues and NTTs; 2 (C) only the FP32
                                  templates are kept and each query encodes the diagonals of every group
                                  on the device before its MAC */
    uint32_t level_mode;       /* 0: the match runs at the query's top level (whole modulus chain);
                                  1: the query is first dropped (limbs discarded) to the lowest level that
                                  still leaves the threshold depth and one output level above 0:
                                  2 + depth with a Chebyshev degree (depth = d2, or d2 + 4 with the hybrid
                                  comparator), 2 without, capped at the top level */
    uint32_t sum_radix;        /* RotateAndSum of the membership result (Algorithm 5's aggregation):
                                  0 or 2: x <- x + Rot_{2^t}(x), one rotation per step (the paper's
                                  power-of-two keys); r = 4, 8, ..., 64: x <- x + sum_{t<r} Rot_{t s}(x)
                                  with s = 1, r, r^2, ..., the r-1 rotations of a step hoisted over one
                                  ModUp (fewer, wider steps; keys t s, see fr_required_rotations). Same
                                  total in every slot, other key-switch noise. */
    uint32_t hoist_giants;     /* on-demand schedule: 0 one ModDown per giant-step rotation (the rotations
                                  of Algorithms 5 and 6 as written); 1 the giant steps of a (query, group)
                                  share one ModDown: their inner products are summed in Q_l u P and
                                  S = P_0 + sum_j sigma_j(P_j.b) + ModDown(sum_j IP_j) (double hoisting,
                                  Section "Hoisting and double hoisting"). Same values, other noise. */
    uint32_t comparator;       /* threshold of FR_MODE_IDENTIFY / FR_MODE_MEMBERSHIP: 0 the paper's GPU
                                  comparator, the degree-n Chebyshev interpolant of step(x - tau) (Eq.
                                  eq:cheb-sign), depth d2; 1 the hybrid comparator of Section "HyDia" (a
                                  Chebyshev approximation followed by a fixed-degree polynomial of Cheon et
                                  al. 2020): y = the degree-n interpolant of sign(x - tau), then
                                  (1 + f_4(y)) / 2 with f_4(y) = (315 y - 420 y^3 + 378 y^5 - 180 y^7 +
                                  35 y^9) / 128, depth d2 + 4. Its slot values are 0 or 1 to within about
                                  1e-2 outside |x - tau| <= 0.02, so a membership sum counts the matches.
                                  level_mode 1 adds the 4 levels to the working level. */
    uint32_t hoist_babies;     /* on-demand schedule, plaintext databases: 0 every baby step B_i = Rot_i(q)
                                  ends with its own ModDown (Algorithm 1's hoisting, the paper's GPU
                                  path); 1 the baby steps stay in Q_l u P before any ModDown (double
                                  hoisting of the baby steps, Section "Hoisting and double hoisting"):
                                  B_i = (P sigma_i(q.b) + IP0_i, IP1_i), the diagonals are kept over
                                  every limb of Q_l u P, and each giant step takes one ModDown of its
                                  sum, fused with its rescale. Same values, other noise; fewer NTTs,
                                  (l + 1 + n_p) / (l + 1) more diagonal words. Encrypted databases
                                  (fr_load_db_encrypted) need 0. */
    uint32_t hoist_sum;        /* RotateAndSum (membership, fr_rotate_sum): 0 every rotation of a step
                                  ends with its own ModDown; 1 the rotations of a step share one ModDown:
                                  their inner products are summed in Q_l u P and x <- x + sum_t
                                  sigma_t(x.b) + ModDown(sum_t IP_t) (double hoisting, Section "Hoisting
                                  and double hoisting", applied to Algorithm 5's aggregation). With
                                  sum_radix 2 it is the radix-2 form bit for bit; with r > 2 the same
                                  total, other noise, one ModDown per step instead of r - 1. */
} fr_params;

/* Set up primes, NTT / base-conversion tables and device state.
 * Errors: FR_ERR_INVALID_ARG (parameters), FR_ERR_CUDA (no device). */
fr_status fr_setup(const fr_params* params, fr_ctx** out);

/* Rotation indices this context needs for `mode` (sorted ascending). Writes at most
 * `cap` entries to `out` and the full count to *n. */
fr_status fr_required_rotations(const fr_ctx* ctx, fr_mode mode, int32_t* out, size_t cap, size_t* n);

/* Rotation-index set of one of the compared schemes (pure host function, no context). */
fr_status fr_rotation_set(uint32_t ell, uint32_t n1, uint32_t slots, fr_keyset which, int membership, int32_t* out,
                          size_t cap, size_t* n);

/* Number of ciphertext rotations a query performs (Section "Complexity analysis of our
 * BSGS-Diagonal"): schedule 0 (grouped, on demand): (n1-1) + G (n2-1); schedule 1
 * (full table, Algorithm 1): ell - 1 (reading: only the ell-1 nontrivial rotations count). */
uint64_t fr_rotation_count(uint32_t ell, uint32_t n1, uint64_t groups, uint32_t schedule);

/* Client-side key generation from a seed (ChaCha20 streams): secret key, public key,
 * relinearisation key and one hybrid key-switching key per rotation index. The secret
 * stays in host memory. */
fr_status fr_keygen(fr_ctx* ctx, const int32_t* rotations, size_t n_rot, uint64_t seed, fr_keys** out);

/* Upload the evaluation keys of `keys` to HBM (resident until fr_free). Only the limbs the
 * context switches are kept: Q limbs 0..working level and the P limbs, in the digits present
 * at that level; key switching above the working level then fails with FR_ERR_LEVEL. */
fr_status fr_load_keys(fr_ctx* ctx, const fr_keys* keys);

/* Load a plaintext template database: row-major K x ell float32 (host pointer),
 * L2-normalised by the caller. Templates are packed per Section "Diagonal method
 * for rectangular matrices" (G = ceil(K / (N/2)) groups) and every pre-rotated
 * diagonal (Eq. eq:prerotation) is encoded on the device and kept in HBM with the
 * limbs of the context's working level (G * ell * (level+1) * N words). */
fr_status fr_load_db(fr_ctx* ctx, const float* templates, size_t K, size_t ell, fr_db** out);

/* Storage tier for the databases loaded from now on (as fr_params.db_tier: 0 auto, 1, 2, 3). */
fr_status fr_set_db_tier(fr_ctx* ctx, uint32_t tier);

/* Encrypted database (the paper's own setting, Section 5.3). fr_encrypt_db is enroller (client)
 * side and runs on the host: for the K x ell FP32 templates (row-major, K >= 1, ell = the
 * context's ell) it writes the G * ell ciphertexts of the diagonals diag_d(M_g), g < G =
 * ceil(K / (N/2)), each encrypted under pk with seed + g*ell + d, to out in the export format
 * ([G][ell][2][level+1][N] u64, coefficient form; words >= G*ell*2*(level+1)*N). With prerotate
 * != 0 the enroller pre-rotates each plaintext diagonal d = j n1 + i by -j n1 slots before
 * encrypting it (Eq. eq:prerotation, the variant of Section 5.3.3; n1 is the context's); with
 * prerotate = 0 the diagonals are plain and the server pre-rotates them at load. The limbs
 * 0..level are those of a top-level encryption with the same seed. Errors: FR_ERR_INVALID_ARG
 * (null pointers, K = 0, ell, small buffer), FR_ERR_LEVEL (level >= number of Q primes). */
fr_status fr_encrypt_db(const fr_ctx* ctx, const fr_keys* keys, const float* templates, size_t K, size_t ell,
                        int prerotate, uint32_t level, uint64_t seed, uint64_t* out, size_t words);
/* Server side: load the G * ell ciphertexts written by fr_encrypt_db (level >= the working
 * level; the limbs above it are dropped) as a database of storage tier 4, resident in HBM in
 * evaluation form. prerotated says how they were enrolled. If 0, the server rotates diagonal
 * j n1 + i, j >= 1, by -j n1 at load (the keys of the negative giant steps -j n1 must be loaded;
 * they are not needed afterwards). Matches take, per group and giant step j, the ct x ct products
 * sum_i Rot_i(q) (x) E_{g, j n1 + i}, relinearise once (lazy relinearisation; the relinearisation
 * key must be loaded), rescale and rotate by j n1; the threshold and the slot sum follow as for
 * plaintext databases. Inputs are copied. Errors: FR_ERR_INVALID_ARG (also a missing key),
 * FR_ERR_LEVEL, FR_ERR_FORMAT (a residue not below its prime), FR_ERR_HBM_BUDGET. */
fr_status fr_load_db_encrypted(fr_ctx* ctx, const uint64_t* cts, size_t K, size_t ell, uint32_t level, int prerotated,
                               fr_db** out);

/* Storage tier chosen for a database (1 stored diagonals, 2 per-query encoding, 3 stored
 * integer coefficients, 4 encrypted diagonals), its number of template groups G = ceil(K / (N/2)), its resident bytes and the BSGS schedule
 * its matches run (0 on demand, 1 table). Any out-pointer may be NULL. */
fr_status fr_db_info(const fr_db* db, uint32_t* tier, uint64_t* groups, uint64_t* bytes, uint32_t* schedule);

/* Client-side encryption of one query q (ell values) replicated across the N/2 slots
 * (numSlots/ell copies, Section "Packed matrices and batched multiplications"). */
fr_status fr_encrypt(const fr_ctx* ctx, const fr_keys* keys, const double* q, size_t ell, uint64_t seed,
                     fr_ct** out);

/* Encrypt an arbitrary slot vector (n = N/2 values) at the top level. */
fr_status fr_encrypt_slots(const fr_ctx* ctx, const fr_keys* keys, const double* z, size_t n, uint64_t seed,
                           fr_ct** out);

/* Encrypted 1:N match of one query (Algorithms 5 and 6). The query must be at the top
 * level; host-resident queries are uploaded (one H2D copy). Returns *n_out library-owned
 * device ciphertexts in *out (array freed with fr_free_cts). */
fr_status fr_match(fr_ctx* ctx, const fr_db* db, const fr_ct* query, fr_mode mode, fr_ct*** out, size_t* n_out);

/* Encrypted match of n_queries (1..64) queries against one database in one pass
 * (configuration "batched launches"): every stage runs once for the whole batch, each
 * rotation key and each plaintext diagonal word is read once for all queries. The
 * outputs of each query equal fr_match's for that query, bit for bit. Returns
 * n_queries * (outputs per query) handles, query after query. */
fr_status fr_match_batch(fr_ctx* ctx, const fr_db* db, const fr_ct* const* queries, size_t n_queries, fr_mode mode,
                         fr_ct*** out, size_t* n_out);

/* Encrypted match of n_queries (1..64) queries, query b against database dbs[b] (configuration
 * "batched launches": many queries against databases of uneven sizes). The baby steps of all
 * queries run as one batch and the giant rotations of each group index as one batch (every
 * rotation key read once per batch); each query's diagonals are multiplied in its own MAC, and
 * a database encoded per query (tiers 2, 3) is encoded once per group for all its queries. The
 * threshold runs on all score ciphertexts at once. Outputs: query after query, G_b each (1 for
 * membership), each query's equal to fr_match's for it, bit for bit. Replayed as a CUDA graph
 * from the second call with the same databases and mode. */
fr_status fr_match_multi(fr_ctx* ctx, const fr_db* const* dbs, const fr_ct* const* queries, size_t n_queries,
                         fr_mode mode, fr_ct*** out, size_t* n_out);

/* ---- Serving loop (continuous batching) ------------------------------------------
 * The paper serves one query at a time (Section "Experimental setup"; the server side of
 * the protocol in Fig. "HyDia protocol"). This loop runs the same match for many clients:
 * fr_match_submit queues a request and returns a ticket at once; a worker thread of the
 * context forms a batch from the oldest request's (database, mode) class (up to max_batch
 * requests of that class in arrival order, a power of two), admits it when one of `slots`
 * streams is free and its workspace fits the HBM left by the batches in flight, and runs
 * it as fr_match_batch would, so batches on different slots overlap on the device while
 * further requests arrive. Each request's outputs equal fr_match's for that query, bit
 * for bit. Keys and databases stay resident. While the loop runs, other calls on the
 * context are serialised with it; a database must stay alive until its requests are
 * polled (fr_free_db waits for the ones in flight). */
typedef struct {
    uint32_t max_batch;        /* 1..64 requests per batch */
    uint32_t slots;            /* 1..8 batches in flight */
    uint64_t hbm_budget_bytes; /* workspace budget of the batches in flight; 0: free HBM at start - 4 GiB */
} fr_serve_params;

/* Start the loop (NULL params: max_batch 8, 2 slots, budget 0). FR_ERR_INVALID_ARG when it
 * already runs. fr_match_submit starts it with the defaults when it is not running. */
fr_status fr_serve_start(fr_ctx* ctx, const fr_serve_params* params);
/* Finish every pending request, then stop the worker; unpolled outputs are freed.
 * fr_free does this first. */
fr_status fr_serve_stop(fr_ctx* ctx);
/* Queue a match request (same arguments and checks as fr_match). The query handle may be
 * freed after the call: host queries are copied (working-level limbs only), device queries
 * share their storage. */
fr_status fr_match_submit(fr_ctx* ctx, const fr_db* db, const fr_ct* query, fr_mode mode, uint64_t* ticket);
/* Outputs of a ticket. block_ms: 0 returns at once, > 0 waits up to that many milliseconds,
 * < 0 waits until done. FR_ERR_TIMEOUT when not finished (the ticket stays valid); on
 * success the ticket is consumed and *out holds *n_out handles (as fr_match). A failed
 * request returns its error once. Unknown tickets: FR_ERR_INVALID_ARG. latency_ms (may be
 * NULL) receives the time from submission to the end of the request's batch on the device
 * (host steady clock, read by a callback the batch's stream runs after its last kernel). */
fr_status fr_match_poll(fr_ctx* ctx, uint64_t ticket, int block_ms, fr_ct*** out, size_t* n_out, double* latency_ms);
/* Requests completed, batches run, requests pending or in flight, and the largest number of
 * batches that were in flight at once. Any out-pointer may be NULL. */
fr_status fr_serve_stats(fr_ctx* ctx, uint64_t* completed, uint64_t* batches, uint64_t* pending,
                         uint64_t* max_concurrent);
/* The loop's batch planner, for inspection: classes[i] is the class of the i-th pending
 * request in arrival order; the next batch takes requests of classes[0]'s class, at most
 * max_batch, rounded down to a power of two, halved while ws_base + B * ws_per_query >
 * avail_bytes. Writes the chosen indices (capacity max_batch) and their count (0: none
 * fits). Host only. */
fr_status fr_serve_plan(const uint32_t* classes, size_t n, uint32_t max_batch, uint64_t avail_bytes,
                        uint64_t ws_base, uint64_t ws_per_query, uint32_t* chosen, size_t* n_chosen);

/* Client-side decryption + decoding of up to n_slots slot values (divided by the nominal scale).
 * At level >= 1 the plaintext is recovered exactly from limbs 0 and 1 (CRT, |m| < q0 q1 / 2). */
fr_status fr_decrypt(const fr_ctx* ctx, const fr_keys* keys, const fr_ct* ct, double* slots, size_t n_slots);

/* Export / import ciphertext words (format above). `words` must be >= 2 (level+1) N. */
fr_status fr_ct_export(const fr_ct* ct, uint64_t* buf, size_t words, uint32_t* level, double* scale);
/* Import copies the words into a host ciphertext of the context: FR_ERR_LEVEL for a level
 * beyond the top, FR_ERR_FORMAT for a residue not below its prime. */
fr_status fr_ct_import(const fr_ctx* ctx, const uint64_t* buf, uint32_t level, double scale, fr_ct** out);
/* Level of a ciphertext and whether it is resident in HBM (either out-pointer may be NULL). */
fr_status fr_ct_info(const fr_ct* ct, uint32_t* level, int* on_device);
/* Move a host ciphertext into HBM (NTT form); no-op if already there. */
fr_status fr_ct_upload(fr_ctx* ctx, fr_ct* ct);

/* Homomorphic primitives on device ciphertexts (paper: GPU primitives mult, add,
 * rotate, rescale; Section "GPU-accelerated encrypted search"). Outputs are new handles. */
fr_status fr_rotate(fr_ctx* ctx, const fr_ct* ct, int32_t k, fr_ct** out);
/* hoisted rotations of one ciphertext by ks[0..n) (one shared ModUp) */
fr_status fr_rotate_hoisted(fr_ctx* ctx, const fr_ct* ct, const int32_t* ks, size_t n, fr_ct** out);
/* Division by the last prime with the centered lift; the level drops by one (FR_ERR_LEVEL at 0). */
fr_status fr_rescale(fr_ctx* ctx, const fr_ct* ct, fr_ct** out);
/* ct x ct product with relinearisation (no rescale); both at the same level */
fr_status fr_mul_relin(fr_ctx* ctx, const fr_ct* a, const fr_ct* b, fr_ct** out);
/* Sum mod q at the lower of the two levels. */
fr_status fr_add(fr_ctx* ctx, const fr_ct* a, const fr_ct* b, fr_ct** out);
/* Threshold of the context (its comparator, degree and tau) on every slot: the Chebyshev
 * interpolant p(x) of step(x - tau) (comparator 0, d2 levels), or the hybrid (1 + f_4(p_sign(x))) / 2
 * (comparator 1, d2 + 4 levels). */
fr_status fr_chebyshev(fr_ctx* ctx, const fr_ct* ct, fr_ct** out);
/* RotateAndSum over all N/2 slots */
fr_status fr_rotate_sum(fr_ctx* ctx, const fr_ct* ct, fr_ct** out);

/* Membership aggregation over parts (Algorithm 5's tail; block-sharded matching): the mod-q
 * sum of the n ciphertexts in parts[] (all at one level), then RotateAndSum over all N/2 slots.
 * Given the FR_MODE_IDENTIFY outputs of every template group of a database -- for example
 * gathered from processes that each hold a range of the groups -- the result is bit-identical to
 * FR_MODE_MEMBERSHIP on the whole database. parts stay owned by the caller; *out is a new
 * handle. FR_ERR_INVALID_ARG for n == 0 or null pointers, FR_ERR_LEVEL for mixed levels. */
fr_status fr_membership_reduce(fr_ctx* ctx, const fr_ct* const* parts, size_t n, fr_ct** out);

/* Rotation by k slots that allocates no device memory (the paper has no counterpart:
 * this is a deployment variant of fr_rotate). For callers that must not allocate
 * while they run -- code captured into a CUDA graph with a fixed memory plan, a
 * serving path that must stay off the allocator, a process whose free HBM belongs
 * to someone else. d_in and d_out are caller-owned device buffers holding one
 * ciphertext in the exported format (coefficient form, [2][level+1][N] uint64);
 * they may not overlap. All temporaries live in one fixed 64 MiB device array
 * inside the library (held by every GPU that loads it until the process exits):
 * calls whose working set needs more (5 (level+1) N + (digits+2)(level+1+n_p) N
 * words; e.g. N=2^16 up to level 8 with 6 digits and 4 special primes) fail with
 * FR_ERR_INVALID_ARG, a level above the loaded keys with FR_ERR_LEVEL, a missing
 * rotation key with FR_ERR_INVALID_ARG; every check runs before anything is
 * enqueued, so a refused call leaves nothing on the stream. The first call on a
 * device looks up the array's device address; make that first call before any
 * stream capture. Every call shares the array, so calls that overlap on the GPU
 * (other streams, other contexts of the same device) race; nothing in it needs to
 * start at zero. Work is enqueued on the context stream. */
fr_status fr_rotate_noalloc(fr_ctx* ctx, const uint64_t* d_in, uint32_t level, int32_t k, uint64_t* d_out);

/* Wait until the device work queued on the context stream has finished. */
fr_status fr_sync(fr_ctx* ctx);

/* Per-region device timing (CUDA events on the context stream). enable=1 clears and
 * starts accumulating, 0 clears and stops; fr_profile_read returns the summed
 * milliseconds, the number of timed launches and their algorithmic bytes (the
 * minimum DRAM reads + writes the launches must make) for a region: "ntt", "modup",
 * "ip", "moddown", "rescale", "tensor", "mac", "encode", "misc", "copy" (device-to-device
 * copies and memsets), the stages "stage:babies", "stage:mac", "stage:giants", "stage:cheb",
 * "stage:sum" and "match". With graphs on (fr_use_graphs, the default) a profiled fr_match /
 * fr_match_batch captures the match with the region events as event-record nodes of a graph
 * and replays it once: regions are timed back to back as in a graph replay, and "match" times
 * the whole replay. With graphs off the events are recorded around each launch as it is
 * enqueued (host launch gaps fall inside the regions). A match profiled by region class runs
 * the two branches of the Chebyshev stage on one stream, so no two regions overlap; one
 * restricted to the stages (fr_profile_only "stage:") keeps the two streams, so "stage:cheb"
 * times the stage as an unprofiled match runs it. The event records add to "match", which
 * therefore exceeds an unprofiled match. */
fr_status fr_profile(fr_ctx* ctx, int enable);
fr_status fr_profile_read(fr_ctx* ctx, const char* region, double* ms, uint64_t* launches, uint64_t* bytes);
/* Restrict profiling to the regions whose name starts with `prefix` (NULL or "": every
 * region); "match" is always timed. Fewer regions mean fewer event records in a profiled
 * replay, so the timed regions run as they do unprofiled. Stays set until changed. */
fr_status fr_profile_only(fr_ctx* ctx, const char* prefix);
/* NTT autotuner (run by fr_setup on device contexts unless the environment sets
 * FR_NTT_TUNE=0): for N >= 2^15 it times each shape of a forward + inverse transform on this
 * GPU for one batch size per bucket (<= 4, <= 16, <= 64, > 64 limb-polynomials; best of 3
 * runs after a warm-up) and keeps the fastest. Shapes 0..3: radix-8 two-pass kernels (8
 * residues per thread), bit 0 = 8 columns per column-pass CTA (else 4), bit 1 = 256-thread
 * row-pass CTAs (else 128); shape 4 (N = 2^16 only): one launch per transform, a cluster of 8
 * CTAs per polynomial exchanging through distributed shared memory; shape 5 (N = 2^16 only):
 * radix-16 two-pass kernels (16 residues per thread, one exchange per pass). shapes[4]
 * receives the chosen shape per bucket, us[24] (may be NULL) the measured microseconds,
 * bucket-major, 6 per bucket (-1: shape not available). */
fr_status fr_ntt_tuning(const fr_ctx* ctx, uint32_t* shapes, double* us);
/* Override the shape per bucket (shapes[4], each 0..5); drops the captured match graphs.
 * Every shape computes the same transform, bit for bit. */
fr_status fr_ntt_set_shapes(fr_ctx* ctx, const uint32_t* shapes);

/* fr_match / fr_match_batch replay a CUDA graph of the whole match from the second call
 * with the same (database, mode, batch size) on (the default). on = 0: every call launches
 * its kernels one by one (the plain per-query form). Results are identical. */
fr_status fr_use_graphs(fr_ctx* ctx, int on);
/* Failure injection (tests of the error paths; host side, no device fault): the after-th
 * stream-ordered device allocation of this context from now on (0: the next one) fails as if
 * HBM were exhausted, so the call that makes it returns FR_ERR_HBM_BUDGET; after < 0 disables
 * it. The context stays usable after the failed call. */
fr_status fr_inject_alloc_failure(fr_ctx* ctx, int64_t after);

/* Device time of the batched negacyclic NTT on this context's ring: npolys limb-polynomials
 * (polynomial p uses prime p mod (level + 1)) transformed forward and inverse on a scratch
 * buffer, each timed with CUDA events on the context stream, best of `reps` after one warm-up
 * round. The shapes in use (fr_ntt_tuning) apply. us_fwd / us_inv receive microseconds per
 * launch sequence (column and row pass). FR_ERR_INVALID_ARG for npolys or reps 0 or null
 * outputs, FR_ERR_LEVEL for a level outside the chain. */
fr_status fr_ntt_time(fr_ctx* ctx, uint32_t npolys, uint32_t level, uint32_t reps, double* us_fwd, double* us_inv);

/* Arithmetic ceiling of the NTT on `device`: forward butterflies (Harvey lazy
 * reduction, Shoup twiddle product, 64-bit residues) per second with every operand in
 * registers, measured by a short microbenchmark. Used as the ALU roofline peak. */
fr_status fr_butterfly_peak(int device, double* butterflies_per_s);
/* FP64 operations per second on `device`: eight independent fused multiply-add chains per
 * thread with register operands, 8 CTAs of 256 threads per SM (an FMA counts as two). The
 * ceiling of the encoder's FP64 special FFT. FR_ERR_CUDA without such a device. */
fr_status fr_fp64_peak(int device, double* flops_per_s);
/* Number of kernel launches issued by the library so far. */
uint64_t fr_launch_count(const fr_ctx* ctx);

/* Context facts: primes (Q then P), digit boundaries, resident HBM bytes. */
fr_status fr_ctx_primes(const fr_ctx* ctx, uint64_t* out, size_t cap, size_t* n);
fr_status fr_ctx_info(const fr_ctx* ctx, uint32_t* n_slots, uint32_t* top_level, uint32_t* n_digits,
                      uint64_t* resident_bytes);
/* Level at which fr_match computes (see fr_params.level_mode). */
uint32_t fr_work_level(const fr_ctx* ctx);

/* Chebyshev coefficients c_0..c_n of the step interpolant (host, no context). */
fr_status fr_cheb_coeffs(uint32_t n, double tau, double* out);
/* The same interpolant of f = 1 for x >= tau and `low` below (low = 0: fr_cheb_coeffs; -1: the
 * sign(x - tau) interpolant the hybrid comparator starts from). */
fr_status fr_cheb_coeffs_lo(uint32_t n, double tau, double low, double* out);

/* Release handles. Free a context's ciphertexts before the context: a device ciphertext
 * returns its memory through it. A database may outlive its context: fr_free releases the
 * database's device memory, and fr_free_db then only releases the handle. Keys do not depend
 * on a context. */
void fr_free_ct(fr_ct* ct);
void fr_free_cts(fr_ct** cts, size_t n);
void fr_free_keys(fr_keys* keys);
void fr_free_db(fr_db* db);
void fr_free(fr_ctx* ctx);
/* Message of the last failed call on this thread (owned by the library). */
const char* fr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FR_H */
