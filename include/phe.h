/*
 * phe.h -- C ABI of libphe, a B300 (sm_103a) engine for the server side of
 * private LoRA fine-tuning under homomorphic encryption (arXiv 2505.07329).
 *
 * The server holds a public int8 weight matrix W (d_out x d_in) in the clear
 * and receives the client's activations x as RLWE ciphertexts, one per block
 * of N coefficients (Sec. 4.3.1: L = ceil(d_in/N) blocks, last one zero
 * padded).  For every token and every output row j it returns the LWE
 * ciphertext of Eq. (LWEdot),
 *
 *     LWE(x . w_j) = sum_{i<L} SampleExtract(RLWE(x_hat_i) . w_hat_ij, N-1),
 *     w_hat_ij[k]  = w_j[iN + N-1-k]                    (reversed weights),
 *
 * followed by the ModulusSwitch to q' = 2^k (Sec. 3.2, Sec. 4.3.1) before the
 * result goes back to the client.  The backward pass computes W^T . [g] with
 * the same primitive (Sec. 6.2: encrypted vector-matrix products in both
 * passes).  The server never sees the secret key (Sec. 5).
 *
 * Conventions
 *   - Every call returns a phe_status; on failure phe_last_error() gives a
 *     message for the calling thread.  Invalid arguments return PHE_EINVAL
 *     and launch nothing.
 *   - Handles (phe_ctx, phe_weights) are opaque, library-owned, and freed
 *     with the matching *_destroy / *_free call.
 *   - Data buffers are caller-owned.  Pointers named d_* are device pointers
 *     on the context's device; h_* are host pointers.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that
 *     take a stream are asynchronous on it unless stated otherwise.
 *   - Ciphertext layout (SoA):
 *       input  mask  A   [T][L][N] uint64, words in [0, q) (larger words are
 *                        reduced mod q on load)
 *       input  body  B   [T][L][N] uint64
 *       output mask  a'  [T][rows][N]  uint32 (switched) or uint64 (raw)
 *       output body  b'  [T][rows]     uint32 (switched) or uint64 (raw)
 *     where rows = d_out for PHE_FWD and d_in for PHE_BWD, and L is formed
 *     from d_in (PHE_FWD) or d_out (PHE_BWD).
 */
#ifndef PHE_H
#define PHE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum phe_status {
    PHE_OK = 0,
    PHE_EINVAL = 1,        /* bad argument, shape or parameter set */
    PHE_ENOMEM = 2,        /* device or host allocation failed */
    PHE_EBUSY = 3,         /* admission refused: capacity in use */
    PHE_ETIMEOUT = 4,      /* a bounded wait ran out */
    PHE_ECUDA = 5,         /* a CUDA runtime call failed */
    PHE_EUNSUPPORTED = 6   /* valid request the build does not support */
} phe_status;

typedef struct phe_ctx phe_ctx;
typedef struct phe_weights phe_weights;

/* Ring and switch parameters (Sec. 3.1 RLWE ciphertexts over
 * R_q = Z_q[X]/(X^N+1); Sec. 3.2 ModulusSwitch q -> q_out).
 *   N          ring degree, a power of two in [256, 8192]
 *   q          ciphertext modulus: either
 *                - a prime 2^53 < q < 2^61 with q = 1 (mod 2N) (e.g. 2^60 - 2^14 + 1;
 *                  rns_p1 = rns_p2 = 0), or
 *                - an RNS modulus 2^53 < q = rns_p1 * rns_p2 < 2^61 of two distinct primes
 *                  below 2^30, each = 1 (mod 2N) (e.g. 1073643521 *
 *                  1073692673); the hot path then runs on 32-bit residues
 *                  and returns to q by the CRT before the switch, or
 *                - a power of two q = 2^K, 8 <= K <= 62, with rns_p1, rns_p2
 *                  as above (the paper's parameter set, Table cryptoparams in
 *                  Sec. 4.4: K = 39, N = 2048, q_out = 2^26).  Products run
 *                  exactly in Z through the residues mod rns_p1 * rns_p2
 *                  (masks lifted to [-2^(K-1), 2^(K-1))), then are reduced
 *                  mod 2^K; this needs N * 127 * 2^(K-1) * L < p1 p2 / 2 for
 *                  the weights' block count L (checked at upload), and the
 *                  switch is a rounding shift (ties up).  No 64-bit form
 *                  and no client encryption for such a q (PHE_EUNSUPPORTED);
 *                  packing holds the key in exact slices (phe_ksk_upload)
 *   log2_qout  k of the output modulus q' = 2^k, 1 <= k <= 32 (k < K for q = 2^K)
 *   flags      PHE_CTX_FORCE_U64: with an RNS modulus, run the 64-bit form
 *              anyway (the results are identical; for cross-checks) */
typedef struct phe_params {
    uint32_t N;
    uint32_t log2_qout;
    uint64_t q;
    uint32_t rns_p1;
    uint32_t rns_p2;
    uint32_t flags;
} phe_params;

#define PHE_CTX_FORCE_U64 1u

#define PHE_FWD 0              /* W   . [x] : rows = d_out, contraction over d_in */
#define PHE_BWD 1              /* W^T . [g] : rows = d_in,  contraction over d_out */
#define PHE_DIR_FWD_BIT 1u
#define PHE_DIR_BWD_BIT 2u

#define PHE_OUT_SWITCHED 0u    /* outputs mod q' = 2^k as uint32 (the protocol's result) */
#define PHE_OUT_RAW 1u         /* outputs mod q as uint64, no switch (testing, unfused use) */
#define PHE_PACK_DENSE 2u      /* packing calls only: several tokens per output RLWE (phe_pack_layout) */

/* Name of a status code.  Never fails. */
const char* phe_status_string(phe_status s);

/* Message of the last failed call made by this thread ("" if none). */
const char* phe_last_error(void);

/* Create a context on CUDA device `device`: validates the parameters
 * (primality, q = 1 mod 2N, bounds), finds a primitive 2N-th root of unity
 * and uploads the twiddle tables.  Blocking.  Errors: PHE_EINVAL for a bad
 * parameter set, PHE_ECUDA if the device is unusable. */
phe_status phe_ctx_create(const phe_params* params, int device, phe_ctx** out);
void phe_ctx_destroy(phe_ctx* ctx);

/* Copy the public weights W (host, int8, row-major [d_out][d_in], caller
 * keeps ownership) to the device and encode them for the directions in
 * `dirs` (PHE_DIR_FWD_BIT | PHE_DIR_BWD_BIT): the reversed blocks w_hat_ij
 * of Sec. 4.3.1, transformed to the NTT domain (and scaled by N^-1), plus a
 * packed int8 copy for the body product.  1 <= d_out, d_in <= 16384.
 * Blocking on `stream`.  Errors: PHE_EINVAL, PHE_ENOMEM, PHE_ECUDA. */
phe_status phe_weights_upload(phe_ctx* ctx, const int8_t* h_W, uint32_t d_out, uint32_t d_in, uint32_t dirs,
                              void* stream, phe_weights** out);
void phe_weights_free(phe_weights* w);

/* Output rows, contraction length and input blocks L for a direction;
 * device bytes held by the handle.  Errors: PHE_EINVAL (direction not
 * uploaded). */
phe_status phe_weights_shape(const phe_weights* w, int dir, uint32_t* rows, uint32_t* cols, uint32_t* L);
uint64_t phe_weights_device_bytes(const phe_weights* w);

/* The hot path, one projection (Eq. (LWEdot) + ModulusSwitch): for T tokens
 * of input ciphertexts (d_in_mask, d_in_body: [T][L][N] uint64) write the T x
 * rows LWE ciphertexts: masks to d_out_mask [T][rows][N] and bodies to
 * d_out_body [T][rows], as uint32 mod 2^k (flags = PHE_OUT_SWITCHED) or as
 * uint64 mod q (flags = PHE_OUT_RAW).  T = 0 is a no-op.
 *
 * The masks run through negacyclic NTTs on the integer ALUs; the bodies
 * b'_tj = sum_k W[j,k] B_t[k] (mod q) run on the tensor cores as an exact
 * bf16 digit GEMM (tcgen05.mma, fp32 accumulation in chunks of 1024 columns,
 * recombined mod q).  Uses stream-ordered scratch of T*L*N*8 bytes
 * (transformed masks) plus 16*T*cols bytes rounded up (the bodies' digit
 * rows), allocated and freed on `stream`.  Every wait inside the tensor-core
 * kernel is bounded: a wait that runs out sets a bit in the context's status
 * word (phe_ctx_status) and that launch's bodies are not written.  Errors:
 * PHE_EINVAL (shapes, null pointers, direction not uploaded), PHE_ENOMEM,
 * PHE_ECUDA. */
phe_status phe_matmul(phe_ctx* ctx, const phe_weights* w, int dir, uint32_t T, const uint64_t* d_in_mask,
                      const uint64_t* d_in_body, void* d_out_mask, void* d_out_body, uint32_t flags, void* stream);

/* Seeded input (Sec. 3.1, "Mask Generation via PRNG"): the client sends a
 * 64-bit seed and the body per ciphertext; the server regenerates the mask.
 * The paper does not name the PRNG; this library reads it as the ChaCha20
 * keystream (RFC 8439) under key = seed (zero-extended), nonce = 0, with
 * coefficient m taken from the 128 bits of words 4(m%4)..4(m%4)+3 of block
 * m/4 (little-endian), reduced mod q.
 *
 * phe_matmul_seeded: as phe_matmul with d_in_seeds [T][L] uint64 in place of
 * the masks; the masks are expanded inside the input transform and never
 * stored.  phe_expand_masks: writes the n masks of d_seeds [n] to
 * d_masks [n][N] (natural order).  Errors: as phe_matmul. */
phe_status phe_matmul_seeded(phe_ctx* ctx, const phe_weights* w, int dir, uint32_t T, const uint64_t* d_in_seeds,
                             const uint64_t* d_in_body, void* d_out_mask, void* d_out_body, uint32_t flags,
                             void* stream);
phe_status phe_expand_masks(phe_ctx* ctx, const uint64_t* d_seeds, uint32_t n, uint64_t* d_masks, void* stream);

/* Unfused ModulusSwitch (Sec. 3.2): out[i] = round(in[i] * 2^k / q) mod 2^k,
 * ties rounded up, for n words (device buffers).  Input words are reduced
 * mod q first.  With an RNS modulus q = p1 p2 the words go through the same
 * residue-form arithmetic as the fused epilogue: residues mod p1 and p2, the
 * CRT digit, then a 32-bit quotient estimate.  Errors: PHE_EINVAL, PHE_ECUDA. */
phe_status phe_modswitch(phe_ctx* ctx, const uint64_t* d_in, uint32_t* d_out, size_t n, void* stream);

/* End-to-end form with HOST buffers: copies the inputs host->device, runs
 * the hot path and copies the results device->host, token chunk by token
 * chunk, so that device memory stays bounded (at most `max_chunk_bytes` of
 * device outputs per chunk; 0 selects 1 GiB).  h_* are host pointers with the
 * same layouts as phe_matmul's device buffers; page-locked host memory makes
 * the copies asynchronous.  Blocking: returns after the last result has
 * reached the host (the stream is synchronized).  Errors: as phe_matmul. */
phe_status phe_matmul_host(phe_ctx* ctx, const phe_weights* w, int dir, uint32_t T, const uint64_t* h_in_mask,
                           const uint64_t* h_in_body, void* h_out_mask, void* h_out_body, uint32_t flags,
                           uint64_t max_chunk_bytes, void* stream);

/* Tracing (for measurement): while enabled, every kernel the library
 * launches with this context is bracketed by CUDA events recorded on the
 * launching stream, and every phe_matmul call by a pair around the whole
 * call.  phe_trace_read waits for the recorded events, fills up to `cap`
 * entries (one per kernel name, plus "phe_matmul" for whole calls) and
 * clears the record.  Not thread-safe: trace one stream at a time.
 * Errors: PHE_EINVAL, PHE_ECUDA. */
typedef struct phe_trace_entry {
    char name[32];
    uint64_t launches;
    double total_ms;
    double p50_ms;
    double p99_ms;
    double max_ms;
} phe_trace_entry;

phe_status phe_trace_enable(phe_ctx* ctx, int on);
phe_status phe_trace_read(phe_ctx* ctx, phe_trace_entry* out, uint32_t cap, uint32_t* n_out);

/* Where the bodies b'_tj = sum_k W[j,k] B_t[k] run (results are identical
 * bit for bit):
 *   PHE_BODY_AUTO    (default) on the tensor cores when a launch group has at
 *                    least 16384 (token, row) outputs, else fused in the mask
 *                    kernel (a dp4a dot product), which has the lower latency
 *                    at one-token sizes;
 *   PHE_BODY_TENSOR  always on the tensor cores;
 *   PHE_BODY_FUSED   always fused (no digit-row scratch).
 * Applies to calls made after it.  Errors: PHE_EINVAL. */
#define PHE_BODY_AUTO 0u
#define PHE_BODY_TENSOR 1u
#define PHE_BODY_FUSED 2u
phe_status phe_ctx_set_body_path(phe_ctx* ctx, uint32_t path);

/* Status word of the context's kernels with bounded waits (the body GEMM):
 * 0 when every wait completed since the last clear; otherwise bit 0 = a
 * tensor-memory operand load, bit 1 = an MMA issue wait, bit 2 = the
 * epilogue's wait, bit 3 = draining copies in flight timed out, and the
 * outputs of that launch are not valid.  Synchronises the device first.
 * clear != 0 resets the word.  Errors: PHE_EINVAL, PHE_ECUDA. */
phe_status phe_ctx_status(phe_ctx* ctx, uint32_t* flags, int clear);

/* Peak probes, run on `device` in the calling process (blocking, a few ms):
 *   phe_probe_alu     register-only Gentleman-Sande butterflies with the
 *                     hot path's own arithmetic, 8 independent chains per
 *                     thread at lwedot's occupancy; form 0 = 32-bit residue
 *                     butterflies (RNS form), 1 = 64-bit butterflies.
 *                     *per_s = butterflies per second (iters 0 = 4096).
 *   phe_probe_tensor  back-to-back tcgen05.mma kind::f16 (bf16, fp32
 *                     accumulate, M 128, N 256, K 16), one CTA per SM;
 *                     *flops_per_s = 2 M N K per MMA per second
 *                     (iters 0 = 20000 rounds of 4 MMAs).
 * They give the denominators of the benchmark's rooflines.  Errors:
 * PHE_EINVAL, PHE_ETIMEOUT (an MMA wait ran out), PHE_ECUDA. */
phe_status phe_probe_alu(int device, int form, uint32_t iters, double* per_s);
phe_status phe_probe_tensor(int device, uint32_t iters, double* flops_per_s);

#ifdef PHE_TESTING
/* ---- Test library only (libphe_test.so, built with -DPHE_TESTING) -------
 * Client-side helpers for tests and benchmarks.  The server never holds the
 * key (Sec. 5): the production libphe.so does not export these calls.
 *
 * phe_test_keygen: a secret key of N coefficients (the context's ring) to
 * host memory h_sk [N] int8, from a 64-bit seed (SplitMix64): kind
 * PHE_KEY_TERNARY draws from {-1, 0, 1}, PHE_KEY_BINARY from {0, 1} (Sec.
 * 3.1 uses a binary key; the workloads here a ternary one).  Host only.
 *
 * phe_client_encrypt: RLWE encryption of T int8 vectors of length d (Sec.
 * 3.1, blocks of Sec. 4.3.1):
 *     B_ti = A_ti * S + E_ti + delta * x_hat_ti  (mod q)
 * d_A [T][L][N] masks in [0, q), d_S [N] int8 key (binary or ternary),
 * d_E [T][L][N] int32 noise, d_x [T][d] int8 messages; writes d_B [T][L][N].
 * Errors: PHE_EINVAL, PHE_ENOMEM, PHE_ECUDA, PHE_EUNSUPPORTED (q = 2^K). */
#define PHE_KEY_BINARY 0u
#define PHE_KEY_TERNARY 1u
phe_status phe_test_keygen(phe_ctx* ctx, uint64_t seed, uint32_t kind, int8_t* h_sk);
phe_status phe_client_encrypt(phe_ctx* ctx, uint32_t T, uint32_t d, const uint64_t* d_A, const int8_t* d_S,
                              const int32_t* d_E, const int8_t* d_x, uint64_t delta, uint64_t* d_B, void* stream);
#endif /* PHE_TESTING */

/* ---- Batched form ------------------------------------------------------
 * Many products at once -- e.g. every projection of a layer in both
 * directions, with uneven token counts -- as one plan.  A plan transforms
 * each distinct input once (products that share d_in_mask, like the q, k and
 * v projections of one x, share the transform) and runs every product's
 * (row, token-chunk) tiles in one persistent lwedot launch per group of up
 * to 32 products.  Buffers are fixed at creation; to process new data, write
 * it into the same input buffers and run the plan again. */
typedef struct phe_job {
    const phe_weights* w;       /* weights (uploaded for `dir`) */
    int32_t dir;                /* PHE_FWD or PHE_BWD */
    uint32_t T;                 /* tokens (0 = skip) */
    const uint64_t* d_in_mask;  /* [T][L][N] */
    const uint64_t* d_in_body;  /* [T][L][N] */
    void* d_out_mask;           /* [T][rows][N] */
    void* d_out_body;           /* [T][rows] */
    const uint64_t* d_in_seeds; /* [T][L] seeds; when not NULL the masks are expanded from them
                                   (see phe_matmul_seeded) and d_in_mask is ignored */
} phe_job;

/* Tile shape of a plan: tokens per (row, token-chunk) tile, and the
 * persistent grid in blocks per SM (0 = one block per tile, not persistent). */
typedef struct phe_tuning {
    uint32_t tok_chunk;
    uint32_t blocks_per_sm;
} phe_tuning;

typedef struct phe_plan_stats {
    uint32_t launches;          /* kernel launches per run */
    uint32_t lwedot_launches;
    uint64_t tiles;
    uint64_t scratch_bytes;     /* transformed inputs held by the plan */
    uint64_t modmuls;           /* algorithmic modular multiplications per run */
    phe_tuning tune;
} phe_plan_stats;

#define PHE_PLAN_MAX_JOBS 1024

typedef struct phe_plan phe_plan;

/* Build a plan over n_jobs products (same output mode `flags` for all);
 * `tune` NULL selects {16 tokens, 3 blocks/SM}.  Allocates the transformed-
 * input scratch (held until phe_plan_destroy).  Errors: PHE_EINVAL (a job's
 * shapes or pointers, too many jobs), PHE_ENOMEM, PHE_ECUDA. */
phe_status phe_plan_create(phe_ctx* ctx, const phe_job* jobs, uint32_t n_jobs, uint32_t flags,
                           const phe_tuning* tune, phe_plan** out);
/* Launch the plan's kernels on `stream` (asynchronous). */
phe_status phe_plan_run(phe_plan* plan, void* stream);
/* The same launches replayed from a CUDA graph: the first call captures
 * them on `stream` (which must not be the legacy default stream) and
 * instantiates the graph; every call launches it (asynchronous).  If tracing
 * is on when the graph is captured, event-record nodes around each lwedot
 * launch are captured too; each replay then adds their timings to the trace
 * (read the trace before replaying the same plan again). */
phe_status phe_plan_graph(phe_plan* plan, void* stream);
phe_status phe_plan_info(const phe_plan* plan, phe_plan_stats* out);
void phe_plan_destroy(phe_plan* plan);

/* Autotuner: times candidate tile shapes (tokens per tile in
 * {2, 4, 8, 16, 32, 64} x persistent or one-block-per-tile grids) on the first
 * `sample_tokens` tokens (0 = 64) of every job, with CUDA events on
 * `stream` (non-default), and returns the fastest.  Writes the jobs' output
 * buffers.  Results are cached per ring and job shapes; a cached answer is
 * returned without timing unless best_ms_per_token is requested.
 * Blocking.  Errors: PHE_EINVAL, PHE_ENOMEM, PHE_ECUDA. */
phe_status phe_autotune(phe_ctx* ctx, const phe_job* jobs, uint32_t n_jobs, uint32_t flags, uint32_t sample_tokens,
                        void* stream, phe_tuning* best, double* best_ms_per_token);

/* ---- Served form ---------------------------------------------------------
 * A server that takes encrypted-matmul requests from many clients and layers
 * as they arrive (continuous batching).  A worker thread runs iterations:
 * each takes the next chunk of `chunk_tokens` tokens of every admitted
 * request that still has tokens, in arrival order, as long as the chunk's
 * device buffers fit `mem_budget_bytes`, and runs them all in one batched
 * launch.  Requests arriving meanwhile join at the next iteration; buffers
 * are reserved per chunk and released when it completes.  Two iterations
 * are kept in flight.  Results of a chunk are copied to the request's host
 * buffers, or dropped when none are given (benchmarking).  Every host wait
 * is bounded by `wait_timeout_ms` (PHE_ETIMEOUT); a failed iteration fails
 * the server and every unfinished request.
 *
 * Admission is FIFO by arrival; a request whose next chunk does not fit the
 * budget may be passed over by younger, smaller ones for at most 4
 * iterations in a row, after which nothing younger is admitted until its
 * chunk fits, so no request waits without bound under sustained load.
 *
 * Failure: after a failed launch or a wait that ran out, no request is
 * admitted any more, and unfinished requests are reported failed (poll -1,
 * wait returns the server's error) only once the work already in flight on
 * the device has drained -- until then that work may still read a request's
 * inputs and write its host buffers.  The server waits for the drain at
 * most max(4 * wait_timeout_ms, 3000) ms; if the device has not drained by
 * then, those requests stay pending (waits time out), and their input and
 * output buffers must stay valid until phe_server_destroy returns, which
 * synchronises the server's stream. */
typedef struct phe_server_config {
    uint64_t mem_budget_bytes;        /* device bytes for in-flight chunk buffers */
    uint32_t chunk_tokens;            /* tokens of one request per iteration */
    uint32_t tok_chunk;               /* tokens per kernel tile */
    uint32_t blocks_per_sm;           /* persistent grid (0 = one block per tile) */
    uint32_t max_active;              /* requests admitted at once */
    uint32_t max_jobs_per_iteration;  /* chunks per iteration */
    uint32_t max_queue;               /* waiting requests before PHE_EBUSY */
    uint32_t wait_timeout_ms;         /* bound on every host wait */
    uint32_t flags;                   /* PHE_OUT_SWITCHED or PHE_OUT_RAW */
    uint32_t simulate;                /* 1: host-only scheduler test backend, no GPU */
    double sim_ns_per_item;           /* simulated cost per (token, row) */
} phe_server_config;

typedef struct phe_request {
    const phe_weights* w;
    int32_t dir;
    uint32_t T;
    const uint64_t* d_in_mask;        /* device [T][L][N], valid until the request completes */
    const uint64_t* d_in_body;
    void* h_out_mask;                 /* host [T][rows][N] (pinned for async copies), or NULL */
    void* h_out_body;                 /* host [T][rows], or NULL */
    uint32_t sim_rows;                /* simulated backend only: output rows */
    const uint64_t* d_in_seeds;       /* [T][L] seeds in place of d_in_mask (NULL: use the masks) */
} phe_request;

typedef struct phe_serving_stats {
    uint64_t submitted, completed, failed, tokens_completed, iterations;
    uint64_t waiting, active, reserved_bytes, peak_reserved_bytes;
    double p50_ms, p99_ms, max_ms, mean_ms;  /* submit -> results complete */
    double busy_ms;                          /* first launch -> last completion */
} phe_serving_stats;

typedef struct phe_server phe_server;

/* Errors: PHE_EINVAL (null or zero sizes), PHE_ECUDA. */
phe_status phe_server_create(phe_ctx* ctx, const phe_server_config* cfg, phe_server** out);
/* Thread-safe, non-blocking.  Errors: PHE_EINVAL, PHE_ENOMEM (one chunk of
 * this request exceeds the budget), PHE_EBUSY (queue full), or the error
 * that failed the server. */
phe_status phe_server_submit(phe_server* srv, const phe_request* req, uint64_t* id);
/* Wait at most timeout_ms for a request (PHE_ETIMEOUT otherwise). */
phe_status phe_server_wait(phe_server* srv, uint64_t id, uint32_t timeout_ms, double* latency_ms);
/* done: 1 complete, 0 pending (or failing, with work still in flight),
 * -1 failed (no work in flight reads or writes its buffers any more). */
phe_status phe_server_poll(phe_server* srv, uint64_t id, int* done, double* latency_ms);
phe_status phe_server_stats(phe_server* srv, phe_serving_stats* out);
/* Drains the admitted and waiting requests, then stops the worker. */
void phe_server_destroy(phe_server* srv);

/* ------------------------------------------------------------------------
 * Output packing (Sec. 3.2 KeySwitching and Rotate; Eq. (pack_rotate); the
 * key-switching products as matrix products, Eq. (gpu_keyswitch), Sec. 4.5)
 *
 * The LWE outputs of rows gN .. gN+m-1 of a token (m = min(N, rows - gN))
 * become one RLWE ciphertext
 *     RLWE_g = ModulusSwitch( sum_{j<m} Rotate(KeySwitching(LWE_{gN+j}), j) ),
 * whose message coefficient j is the message of output row gN+j (zero for
 * j >= m).  This replaces rows*(N+1) words per token by G*2N,
 * G = ceil(rows/N).
 *
 * Dense packing (flags | PHE_PACK_DENSE; not in the paper, which packs one
 * token's outputs per RLWE): for rows <= N/2, the outputs of tpu =
 * floor(N/rows) consecutive tokens share one RLWE, token t's row r at
 * coefficient (t mod tpu)*rows + r of RLWE floor(t/tpu); the last RLWE holds
 * the remaining T mod tpu tokens (if any) and zeros past them.  The same sum
 * of Eq. (pack_rotate) over a longer list of LWE ciphertexts: ceil(T/tpu)
 * RLWEs instead of T, and as many fewer key-switching contractions.  For
 * rows > N/2 the flag changes nothing.  Output buffers hold units*N words
 * (phe_pack_layout), unit-major.
 *
 * KeySwitching of (a, b) under the LWE key s (dimension n = N: the RLWE key's
 * coefficients, as SampleExtract leaves them) to the RLWE key S' is
 *     (A', B') = (0, b) - sum_{i<n} sum_{l<ell} d_l(a_i) KSK_{i,l},
 * with Decomp read as the approximate signed gadget decomposition: a~ is the
 * ModulusSwitch of a to B^ell (B = 2^base_log), d_0 .. d_{ell-1} are its
 * signed base-B digits in [-B/2, B/2) (d_0 most significant), and KSK_{i,l}
 * encrypts the constant polynomial s_i round(q / B^(l+1)) under S'.
 * ------------------------------------------------------------------------ */
typedef struct phe_ksk phe_ksk;

/* Copies a key-switching key to the device and precomputes its NTT form
 * (-N^-1 NTT(KSK) with Shoup quotients; 2*n*ell*N*16 bytes).
 *   h_ka, h_kb  host [n][ell][N] uint64: KSK_{i,l} = (h_ka[i][l], h_kb[i][l]),
 *               words mod q (larger words are reduced); caller keeps them.
 *   n           LWE dimension; must equal N.
 *   base_log, ell  1 <= ell <= 4, 1 <= base_log <= 30, base_log*ell <= 32;
 *               with an RNS modulus also 2^(base_log-1) < min(p1, p2).
 * With q = 2^K (computed through p1 p2) the contraction has no NTT mod q, so
 * it runs exactly over the integers through p1 p2.  The centred key is split
 * into S balanced slices of b bits, KSK = sum_s 2^(b s) KSK_s, with b the
 * largest width such that n*ell*N*(B/2)*2^(b-1) < p1 p2 / 2 and
 * S = ceil((K+1)/b) <= 8.  The device copy is S times larger, and the
 * contraction runs once per slice.
 * Synchronous.  Errors: PHE_EINVAL (shape or parameters), PHE_EUNSUPPORTED
 * (q = 2^K with no exact slice width), PHE_ENOMEM, PHE_ECUDA. */
phe_status phe_ksk_upload(phe_ctx* ctx, const uint64_t* h_ka, const uint64_t* h_kb, uint32_t n, uint32_t base_log,
                          uint32_t ell, phe_ksk** out);
void phe_ksk_free(phe_ksk* k);
uint64_t phe_ksk_device_bytes(const phe_ksk* k);

/* Output RLWEs (units) of T tokens of `rows` outputs each at ring degree N,
 * and the tokens each packs (1 unless flags has PHE_PACK_DENSE and
 * 2*rows <= N).  Host only.  Errors: PHE_EINVAL (N not a power of two,
 * rows = 0, unknown flags). */
phe_status phe_pack_layout(uint32_t N, uint32_t rows, uint32_t T, uint32_t flags, uint64_t* units,
                           uint32_t* tokens_per_unit);

/* Packs T x rows given LWE ciphertexts of dimension N.
 *   d_lwe_mask  [T][rows][N] uint64 words below q (as phe_matmul writes with PHE_OUT_RAW;
 *               larger words give unspecified results, never a fault); 16-byte aligned
 *   d_lwe_body  [T][rows]    uint64 mod q
 *   d_out_a, d_out_b  [T][G][N]: uint32 words mod 2^log2_qout (PHE_OUT_SWITCHED)
 *               or uint64 mod q (PHE_OUT_RAW); RLWE_g of token t at (t*G + g)*N.
 *               With PHE_PACK_DENSE: [units][N] (phe_pack_layout).
 * Allocates its scratch (at most 4 GiB of digit rows at a time) on `stream`
 * from the context's memory pool.  Errors: PHE_EINVAL (handles, flags,
 * more than 2^24 output RLWEs, unaligned masks), PHE_ENOMEM, PHE_ECUDA. */
phe_status phe_pack(phe_ctx* ctx, const phe_ksk* k, uint32_t T, uint32_t rows, const uint64_t* d_lwe_mask,
                     const uint64_t* d_lwe_body, void* d_out_a, void* d_out_b, uint32_t flags, void* stream);

/* The paper's whole server path, Eq. (LWEdot) then Eq. (pack_rotate), token
 * chunk by token chunk: the product kernel switches the LWE masks straight to
 * the gadget modulus B^ell (all that Decomp reads) and keeps the bodies mod
 * q, in a scratch buffer of at most 2 GiB (or one unit's tokens, if more),
 * then the packing runs on them.  The result equals phe_matmul (PHE_OUT_RAW)
 * followed by phe_pack with the same flags.  Inputs as phe_matmul; outputs
 * and flags (PHE_OUT_RAW, PHE_PACK_DENSE) as phe_pack with rows of
 * direction `dir`. */
phe_status phe_matmul_packed(phe_ctx* ctx, const phe_weights* w, const phe_ksk* k, int dir, uint32_t T,
                             const uint64_t* d_in_mask, const uint64_t* d_in_body, void* d_out_a, void* d_out_b,
                             uint32_t flags, void* stream);

/* phe_matmul_packed with seeded input masks (as phe_matmul_seeded). */
phe_status phe_matmul_packed_seeded(phe_ctx* ctx, const phe_weights* w, const phe_ksk* k, int dir, uint32_t T,
                                    const uint64_t* d_in_seeds, const uint64_t* d_in_body, void* d_out_a,
                                    void* d_out_b, uint32_t flags, void* stream);

/* phe_matmul_packed with HOST buffers, `tok_chunk` tokens at a time (0
 * selects 8; with PHE_PACK_DENSE rounded down to whole units, at least
 * one): inputs host->device, the packed path, packed outputs
 * device->host, double-buffered on two streams.  h_* have the layouts of the
 * device buffers above; page-locked host memory makes the copies
 * asynchronous.  Blocking: returns after the last result has reached the
 * host.  Errors: as phe_matmul_packed. */
phe_status phe_matmul_packed_host(phe_ctx* ctx, const phe_weights* w, const phe_ksk* k, int dir, uint32_t T,
                                  const uint64_t* h_in_mask, const uint64_t* h_in_body, void* h_out_a,
                                  void* h_out_b, uint32_t flags, uint32_t tok_chunk, void* stream);

/* ------------------------------------------------------------------------
 * Wire format (Sec. 4.4: the sizes of the client's and the server's
 * messages; Sec. 4.5: the result goes back "packed into a bit-vector").
 * A record is a little-endian bit stream of fixed-width fields: field m of
 * width b occupies stream bits m*b .. m*b+b-1, stream bit j is bit j%8 of
 * byte j/8, and the record is zero-padded to a multiple of 32 bits (4-byte
 * aligned records).
 *   input record  8-byte seed (little endian), then the N body words of one
 *                 block at ceil(log2 q) bits (Sec. 3.1: the mask is
 *                 regenerated from the seed); N = 2048, q = 2^39: 9992 bytes
 *   LWE record    the N mask words, then the body, at log2_qout bits
 *   RLWE record   A then B (2N words) at log2_qout bits; N = 2048 at 26 bits
 *                 gives the 13312 bytes of Sec. 4.4
 * ------------------------------------------------------------------------ */

/* Record sizes in bytes for the context (any pointer may be NULL). */
phe_status phe_wire_sizes(const phe_ctx* ctx, uint64_t* in_record, uint64_t* lwe_record, uint64_t* rlwe_record);

/* Packs n_records records of fa words from d_a (record r at d_a + r*fa) then
 * fb words from d_b (at d_b + r*fb), each taken mod 2^log2_qout, into
 * consecutive records of 4*ceil((fa+fb)*log2_qout/32) bytes at d_out.
 * Device buffers.  Errors: PHE_EINVAL, PHE_ECUDA. */
phe_status phe_wire_pack(phe_ctx* ctx, const uint32_t* d_a, uint32_t fa, const uint32_t* d_b, uint32_t fb,
                         uint64_t n_records, void* d_out, void* stream);

/* Unpacks n_records consecutive input records (4-byte aligned) into d_seeds
 * [n_records] and d_bodies [n_records][N].  Errors: PHE_EINVAL, PHE_ECUDA. */
phe_status phe_wire_unpack_inputs(phe_ctx* ctx, const void* d_records, uint64_t n_records, uint64_t* d_seeds,
                                  uint64_t* d_bodies, void* stream);

/* The server call on wire records: T*L input records (token-major, block
 * minor) in; out, with k == NULL, T*rows LWE records (phe_matmul_seeded's
 * switched outputs), or with a key-switching key, T*ceil(rows/N) RLWE records
 * (phe_pack's outputs).  Allocates its scratch (at most 2 GiB per token
 * chunk) on `stream`.  Errors: as phe_matmul_seeded and phe_pack. */
phe_status phe_matmul_wire(phe_ctx* ctx, const phe_weights* w, const phe_ksk* k, int dir, uint32_t T,
                           const void* d_in_records, void* d_out_records, void* stream);

/* Size of the fixed device scratch array used by phe_matmul_noalloc. */
#define PHE_NOALLOC_MAX_SCRATCH_BYTES (16u << 20)

/* phe_matmul without any allocation.  The paper has no counterpart: this is
 * an engineering variant for callers that cannot allocate device memory
 * while serving -- e.g. a process whose HBM is already owned by another
 * allocator (a PyTorch caching allocator, an inference server with a fixed
 * budget), where an allocation by this library could fail or fragment that
 * budget, or a latency-critical loop that must not touch the CUDA allocator
 * after start-up.
 *
 * Same arguments, layouts and results as phe_matmul.  The scratch it needs
 * (the transformed input masks, T*L*N*8 bytes) lives in one fixed device
 * array of PHE_NOALLOC_MAX_SCRATCH_BYTES (16 MiB) that every GPU loading the
 * library holds until the process exits; larger requests return PHE_EINVAL
 * (at N = 4096, L = 1: up to 512 tokens per call).  It calls no cudaMalloc,
 * cudaFree or other allocating routine and records no trace events.
 *
 * phe_ctx_create loads the array on its device (with that device current),
 * so its memory is reserved when a context is set up, never inside this
 * call.  Each call looks up the array's address in the current CUDA context
 * (cudaGetSymbolAddress, which allocates nothing once the array is loaded),
 * so a device reset or another context does not leave a stale address.
 * Unlike phe_matmul, the bodies are computed by a dot product fused into the
 * mask kernel (no tensor-core digit rows, which would need more scratch);
 * the results are the same bit for bit.  All calls share the one array
 * and it keeps the last call's contents (each call overwrites every word it
 * reads, so nothing needs clearing): calls whose work overlaps on the GPU --
 * concurrent streams, or several host threads -- race on it and must be
 * serialised by the caller.  Errors: as phe_matmul, plus PHE_EINVAL when the
 * scratch does not fit. */
phe_status phe_matmul_noalloc(phe_ctx* ctx, const phe_weights* w, int dir, uint32_t T, const uint64_t* d_in_mask,
                              const uint64_t* d_in_body, void* d_out_mask, void* d_out_body, uint32_t flags,
                              void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PHE_H */
