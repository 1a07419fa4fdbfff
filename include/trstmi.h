/*
 * trstmi.h -- C ABI of the GB300 (sm_103a) TRSTMI coherence-search library.
 *
 * The library searches for complex frames Phi in C^{d x N} with unit-norm
 * columns and low coherence mu(Phi) = max_{j != k} |<phi_j, phi_k>|
 * (arXiv 2207.06374, Sec. "Introduction", definition of mu_{N,d}).  Each
 * iteration of the stochastic trust-region search scores K random candidates
 *     Phi_c = normalise_columns(Phi + Delta * Z_{t,c}),  Z ~ CN(0,1) entrywise
 * by their exact coherence, keeps the best one if it lowers mu, and expands or
 * contracts the trust radius Delta (the Monte-Carlo sampling and trust-region
 * framework of Sec. "Optimization procedure"; the candidate step and the radius
 * rule are this library's reading of that section, stated with each field).
 *
 * Conventions
 *   - Every function returns an int status: TRSTMI_OK (0), TRSTMI_PENDING (1)
 *     or a negative error code; trstmi_strerror() names it.
 *   - Frames crossing the ABI are HOST buffers owned by the caller: 2*d*N
 *     doubles, column-major with interleaved (re, im), i.e. element (i, j) at
 *     [2*(j*d + i)] (real) and [2*(j*d + i) + 1] (imaginary).
 *   - Handles are opaque and owned by the library.  One handle must not be
 *     used from two threads at once.
 *   - All device work is issued on the stream given in the options (NULL =
 *     a stream the library creates); calls that return host data synchronise
 *     that stream.  There is no CPU fallback: without a usable CUDA device
 *     every call that needs one returns TRSTMI_ECUDA.
 */
#ifndef TRSTMI_H
#define TRSTMI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- statuses */
#define TRSTMI_OK 0
#define TRSTMI_PENDING 1
#define TRSTMI_EINVAL (-1)       /* bad argument (sizes, NULL pointers, options) */
#define TRSTMI_ENOMEM (-2)       /* device allocation failed or budget exceeded */
#define TRSTMI_ECUDA (-3)        /* CUDA runtime error or no device */
#define TRSTMI_ETIMEOUT (-4)     /* a device-side wait hit its time limit */
#define TRSTMI_ECANCELLED (-5)   /* request cancelled */
#define TRSTMI_EBUSY (-6)        /* queue full */
#define TRSTMI_EUNSUPPORTED (-7) /* shape/precision combination not built */
#define TRSTMI_ENOTFOUND (-8)    /* unknown ticket */
#define TRSTMI_ESIZE (-9)        /* size beyond a fixed built-in limit */

/* ----------------------------------------------------- precision modes */
typedef enum trstmi_precision {
  /* candidates generated, scored and accepted in binary64 */
  TRSTMI_FP64 = 0,
  /* complex64 storage, binary32 Gram; acceptance on the binary32 mu */
  TRSTMI_FP32 = 1,
  /* candidates screened by a bf16 tensor-core Gram (fp32 accumulation), the
     top-k survivors re-scored in binary32, the best survivor regenerated,
     renormalised and certified in binary64; acceptance on the binary64 mu */
  TRSTMI_BF16_SCREEN = 2,
  /* as TRSTMI_BF16_SCREEN with fp16 screen operands: same tensor rate and
     storage, unit roundoff 2^-11 instead of 2^-8 (screen error on mu at most
     2u + u^2 for unit columns: 9.8e-4 instead of 7.8e-3; measured on random
     frames with d >= 2: below 1e-3 and 4e-3) */
  TRSTMI_FP16_SCREEN = 3,
  /* as TRSTMI_BF16_SCREEN with tf32 screen operands (fp32 values rounded to
     10 mantissa bits; kind::tf32 MMAs at half the bf16 tensor rate, twice the
     shared memory per column block: the screen takes N <= 768) */
  TRSTMI_TF32_SCREEN = 4
} trstmi_precision;

/* ---------------------------------------------------------- options */
typedef struct trstmi_options {
  int32_t K;            /* candidates per iteration (default 256), >= 1 */
  int32_t precision;    /* trstmi_precision (default TRSTMI_FP64) */
  int32_t topk;         /* BF16_SCREEN: survivors re-scored in fp32 (default 8, 1..64) */
  int32_t trace_cap;    /* rows of the per-iteration trace ring (default 4096, >= 0) */
  double delta0;        /* initial trust radius (default 0.1), > 0 */
  double gamma_inc;     /* radius factor on accept (default 2.0), >= 1 */
  double gamma_dec;     /* radius factor on reject (default 0.25), in (0, 1] */
  double delta_min;     /* radius floor (default 1e-9) */
  double delta_max;     /* radius cap (default 1.0) */
  double target_mu;     /* stop once mu <= target_mu (default 0 = never) */
  /* screen modes: an iteration ranks its candidates with the tensor-core
     screen while its radius is >= screen_min_delta, and with the binary32
     Gram of every candidate below it, where candidate coherences differ by
     less than the screen's resolution (default 0.01; 0 = always screen).
     The screen takes d <= 32 (bf16, fp16, tf32) and 32 < d <= 64 (bf16,
     fp16: two 128-byte operand atoms per column), 2 <= N <= 65536: up to
     1536 columns (768 with two atoms) a candidate's blocks stay resident,
     beyond that it is swept in bands of 1280 (512) columns whose right-hand
     blocks stream through the shared memory.  Other shapes always rank with
     the binary32 Gram; the re-score and certification are unchanged. */
  double screen_min_delta;
  void *stream;         /* cudaStream_t to issue on, or NULL */
  int32_t device;       /* CUDA device ordinal (default 0) */
  int32_t reserved0;
  /* Device memory (default NULL: cudaMalloc / cudaFree).  With dev_alloc
     set, every device allocation of a handle made from these options --
     the instance's state block and the temporary buffers of trstmi_score
     and trstmi_profile_score, the batch's arena, launch plan and candidate
     scratch, the server's control tables, arena, launch plan and candidate
     scratch -- is dev_alloc(bytes, alloc_ctx), released by
     dev_free(ptr, alloc_ctx) (both must be set).  The library calls them on
     the thread that calls it (for a server: trstmi_server_create and
     trstmi_server_destroy), with the handle's device current; dev_alloc
     returns memory of that device, 256-byte aligned, or NULL, which the
     call reports as TRSTMI_ENOMEM.  Memory is released only after the
     handle's stream has finished with it.  A caching allocator (PyTorch's,
     from the Python binding) can serve both. */
  void *(*dev_alloc)(size_t bytes, void *alloc_ctx);
  void (*dev_free)(void *ptr, void *alloc_ctx);
  void *alloc_ctx;
} trstmi_options;

/* Fills *opt with the defaults listed above. */
void trstmi_default_options(trstmi_options *opt);

typedef struct trstmi_instance *trstmi_handle;

/* One row per iteration (binary64 values are mu^2, not mu). */
typedef struct trstmi_trace_row {
  uint32_t t;           /* iteration counter (1-based) */
  uint32_t cstar;       /* chosen candidate index */
  double mu2_best;      /* mu^2 of the chosen candidate in the deciding precision */
  double mu2_screen;    /* its screen (bf16) or fp32 score; = mu2_best otherwise */
  double mu2_cur;       /* mu^2 of the current frame after the decision */
  double delta_used;    /* radius the candidates were drawn with */
  double delta_next;    /* radius after the update */
  int32_t accepted;     /* 1 if the candidate replaced the frame */
  int32_t flags;        /* bit 0: candidates ranked by the tensor-core screen;
                           bit 1 (screen modes): the best survivor was rejected on
                           its binary32 mu^2, which exceeded the current mu^2 by
                           more than twice the fp32/fp64 error bound
                           2 (2d + 18) 2^-24, so the exact rule rejects it too; no
                           binary64 certification ran and mu2_best holds that
                           binary32 value; bit 2: the certification's pair list
                           overflowed and the binary64 pass covered every pair */
} trstmi_trace_row;

typedef struct trstmi_step_info {
  int32_t iters_done;   /* iterations run by this call */
  int32_t accepts;      /* accepted candidates in this call */
  double mu;            /* mu of the current frame (deciding precision) */
  double delta;         /* current radius */
  uint64_t pairs_scored;/* K * N(N-1)/2 per iteration run (screen pairs in BF16 mode) */
  uint64_t elapsed_ns;  /* device time of the call (CUDA events) */
  int32_t done;         /* 1 once mu <= target_mu */
  int32_t reserved;
} trstmi_step_info;

/*
 * Creates a search instance for N >= 2 columns in C^d, d >= 1 (N <= d is
 * allowed; its optimum is mu = 0).  Allocates the device state, draws the
 * seeded initial frame (Algorithm "TRSTMI optimization steps", step 1: random
 * unit vectors; Philox counter tag 1) and scores it in the deciding precision.
 * opt may be NULL for the defaults.  On error *out is set to NULL.
 */
int trstmi_create(int N, int d, uint64_t seed, const trstmi_options *opt,
                  trstmi_handle *out);

/*
 * Runs up to iters >= 0 iterations (fewer if mu reaches target_mu).  Issues
 * them as replays of a captured CUDA graph with no host synchronisation
 * between iterations; synchronises the stream once at the end.  info may be
 * NULL.
 */
int trstmi_step(trstmi_handle h, int iters, trstmi_step_info *info);

/* ------------------------------------------------ candidate sharding
 * One search spread over G processes (one GPU each): the K candidates of an
 * iteration are independent and each is a pure function of (seed, t, c, Phi)
 * (Sec. "Optimization procedure", Monte-Carlo sampling of the trust region),
 * so rank r scores its own range c_lo .. c_hi-1 and the ranks exchange only
 * the K-entry score vector.  An iteration on every rank is:
 *
 *   trstmi_shard_score(h, c_lo, c_hi, scores);    scores: device, K entries
 *   element-wise MAX all-reduce of scores over the ranks (caller: NCCL,
 *     torch.distributed, ...; entries are non-negative, so signed integer
 *     MAX of the bit patterns is exact)
 *   trstmi_shard_finish(h, scores, info);
 *
 * Every rank holds the same state (same N, d, seed and options, same calls),
 * takes the same decisions from the reduced vector and keeps an identical
 * frame; the result is bit-identical to trstmi_step on one GPU.  In the
 * screen modes the top-k re-score and the binary64 certification run on
 * every rank (they are a small part of the iteration).
 */

/* Bytes of the score vector: K x 4 (uint32 bit patterns of the binary32
 * scores: TRSTMI_FP32 and the screen modes) or K x 8 (binary64 bit patterns:
 * TRSTMI_FP64). */
int trstmi_shard_score_bytes(trstmi_handle h, size_t *bytes);

/* Starts the next iteration and writes the ranking score of candidates
 * c_lo .. c_hi-1 (0 <= c_lo <= c_hi <= K) into the caller's device array
 * scores (trstmi_shard_score_bytes bytes), zero everywhere else.  The copy is
 * ordered on the instance's stream; with a library-owned stream the call
 * returns after it completed.  TRSTMI_EINVAL on a bad range or NULL. */
int trstmi_shard_score(trstmi_handle h, int c_lo, int c_hi, void *scores);

/* Completes the iteration started by trstmi_shard_score from the reduced
 * score vector (device, read on the instance's stream: when the exchange ran
 * on another stream the caller orders or synchronises it first); info as in
 * trstmi_step for one iteration.  Synchronises the stream. */
int trstmi_shard_finish(trstmi_handle h, const void *scores, trstmi_step_info *info);

/*
 * Certified coherence of the current frame: the frame is renormalised in
 * binary64 and mu computed in binary64 over all pairs j < k (a binary32
 * pass preselects the pairs within its rounding-error bound of the max, the
 * maximum over those is taken in binary64 -- exact by that bound).
 * welch (nullable) receives sqrt((N-d)/(d(N-1))) (Sec. "Welch bound and
 * equiangular lines"), 0 for N <= d.
 */
int trstmi_coherence(trstmi_handle h, double *mu, double *welch);

/* Copies the current binary64 frame to out (2*d*N doubles, host). */
int trstmi_get_phi(trstmi_handle h, double *out);

/* Replaces the frame (host buffer, 2*d*N doubles); columns are renormalised
 * in binary64 and the frame rescored.  A zero or non-finite column is
 * TRSTMI_EINVAL (checked on the host; the frame is then unchanged).  Returns
 * once `in` has been read: the renormalisation and the rescore are enqueued on
 * the handle's stream ahead of any later call's work, and a device error they
 * meet is reported by the next call that reads the state. */
int trstmi_set_phi(trstmi_handle h, const double *in);

/*
 * Checkpoint: the whole search state (frame, radius, iteration counter,
 * current mu, accept count, options, seed) as a self-describing blob.  With
 * blob == NULL, *size receives the size needed.  Because every random draw
 * is a pure function of (seed, t, c), restoring a blob and running m
 * iterations gives bit-identical results to running them without the
 * interruption.
 */
int trstmi_get_state(trstmi_handle h, void *blob, size_t *size);
int trstmi_set_state(trstmi_handle h, const void *blob, size_t size);

/* Copies the last min(n, trace_cap, iterations run) trace rows, oldest
 * first, to rows; *n_out receives the count. */
int trstmi_get_trace(trstmi_handle h, trstmi_trace_row *rows, int n, int *n_out);

/* Frees everything.  Safe on NULL. */
void trstmi_destroy(trstmi_handle h);

/* Static string for a status code. */
const char *trstmi_strerror(int status);

/* Detail of the last CUDA failure seen by the calling thread (the CUDA error
 * name and text and the failing call), "" if none.  Valid until the thread's
 * next failing call. */
const char *trstmi_last_error(void);

/* ------------------------------------------------------- batched searches
 * Many independent searches of different (N, d) advanced together: each
 * iteration is one set of shared launches over all of them (a persistent
 * scoring pass whose CTAs take (instance, candidate, tile) work items from a
 * counter, one CTA per instance for the accept rule and the commit),
 * replayed from a captured CUDA graph.  Each instance keeps its own state,
 * seed and counters and follows exactly the trajectory that trstmi_create +
 * trstmi_step would give it alone (same options).  Tile widths (16, 32 or 64
 * columns) are chosen per (d, ceil log2 N) by an autotuner that times the
 * scoring pass on the instances themselves at creation; choices are cached
 * for the process.  Every precision mode is accepted; in the screen modes the
 * tensor-core screen of every instance it takes runs as one shared launch per
 * operand format (d <= 32, and 32 < d <= 64) over all (instance, candidate)
 * pairs, then re-score, certification, accept rule and commit run as shared
 * launches too.  Outside binary64, the candidate passes of large instances
 * (N >= 384, scored in tiles) draw each candidate once into a scratch and run
 * the double-buffered tile pass, one such instance after the other; the
 * scratch holds the largest such instance's candidates (at most 512 MiB) and
 * is allocated at creation.
 */
typedef struct trstmi_batch *trstmi_batch_handle;

/* n instances, N[i] >= 2, 1 <= d[i] <= 256, seeds[i]; options shared (K,
 * precision, radius rule, target, trace_cap, stream, device). */
int trstmi_batch_create(int n, const int *N, const int *d, const uint64_t *seeds,
                        const trstmi_options *opt, trstmi_batch_handle *out);
/* Up to iters iterations for every instance (an instance stops early at its
 * target).  info (nullable) aggregates: iters_done = max over instances,
 * accepts and pairs_scored = sums, mu = max over instances, done = all done. */
int trstmi_batch_step(trstmi_batch_handle b, int iters, trstmi_step_info *info);
/* mu of every instance in the deciding precision (n doubles, host) and, if
 * iters is not NULL, the iterations each has run. */
int trstmi_batch_mu(trstmi_batch_handle b, double *mu, int32_t *iters);
/* Binary64 frame of instance i (2*d*N doubles, host). */
int trstmi_batch_get_phi(trstmi_batch_handle b, int i, double *out);
/* Trace rows of instance i, as trstmi_get_trace. */
int trstmi_batch_get_trace(trstmi_batch_handle b, int i, trstmi_trace_row *rows, int n,
                           int *n_out);
/* Tile width (columns) the autotuner chose for every instance (n ints). */
int trstmi_batch_tile_widths(trstmi_batch_handle b, int *widths);
/* Measurement: mean device time of one ranking pass over all instances (the
 * persistent scoring launches of one iteration, or in the screen modes the
 * shared tensor-core screen launch, bracketed by CUDA events; flush_bytes of
 * scratch rewritten before each, outside the events).  Does not advance any
 * instance. */
int trstmi_batch_profile_score(trstmi_batch_handle b, int launches, size_t flush_bytes,
                               double *avg_ms);
/* Frees everything.  Safe on NULL. */
void trstmi_batch_destroy(trstmi_batch_handle b);

/* --------------------------------------------------------- multi-start
 * The paper repeats its procedure for L random initialisations and returns
 * the minimum over the trials (Algorithm "TRSTMI optimization steps", last
 * step; its experiments use L = 2 d^2).  Trial i is the search with seed
 * seed0 + i, run for iters iterations with the given options exactly as
 * trstmi_create + trstmi_step would run it alone; the trials are advanced
 * as batched instances, at most batch_cap per batch (<= 0: all at once),
 * which does not change any result.
 */
typedef struct trstmi_multistart_result {
  double mu;            /* min over the trials of mu (deciding precision) */
  int32_t best;         /* trial reaching it (lowest index on ties) */
  int32_t trials;       /* L used */
  uint64_t best_seed;   /* seed0 + best */
} trstmi_multistart_result;

/* L <= 0 selects 2*d*d trials.  mu_all (nullable, host): L doubles, every
 * trial's mu.  best_phi (nullable, host): 2*d*N doubles, the winning trial's
 * binary64 frame.  Returns the batch or search errors (TRSTMI_EINVAL for bad
 * shapes or options). */
int trstmi_multistart(int N, int d, uint64_t seed0, int L, int iters,
                      const trstmi_options *opt, int batch_cap,
                      trstmi_multistart_result *out, double *mu_all, double *best_phi);

/* ------------------------------------------------------------- serving
 * A persistent request loop on one GPU.  A host scheduler thread keeps up to
 * max_slots searches resident (frame, radius, counters and random-stream
 * position stay on the device) and advances all of them together: each round
 * is iters_per_round iterations of the shared batched launches.  Requests
 * wait in a FIFO queue; the head is admitted as soon as a slot and its device
 * memory fit within hbm_budget (continuous batching: requests that arrive
 * while others run join at the next round).  A search retires at a round
 * boundary once it reached its target, spent its iteration budget or was
 * cancelled.  Every search keeps its own state, so its result is exactly the
 * one trstmi_create + trstmi_step give alone with the same options, seed and
 * budget.  Every precision mode is accepted; in the screen modes each slot
 * also holds its top-k, certification scratch and a pair list of up to 65536
 * pairs,
 * and the slot's device memory grows accordingly.
 */
typedef struct trstmi_server trstmi_server;

typedef struct trstmi_server_opts {
  trstmi_options search;   /* options of every search (K, precision, radius rule,
                              trace_cap, device, stream); target_mu comes from
                              the request */
  size_t hbm_budget;       /* bytes of device memory for resident searches (default 4 GiB);
                              outside binary64, min(1/8, 256 MiB) of it is the scratch in
                              which the candidates of large searches (N >= 384) are
                              drawn once per pass */
  int32_t max_slots;       /* resident searches at most (default 256) */
  int32_t iters_per_round; /* iterations per shared round (default 20) */
  int32_t queue_cap;       /* queued requests at most; beyond: TRSTMI_EBUSY (default 65536) */
  int32_t reserved;
  /* resident work cap: the queue head is admitted only while the resident
     searches' pairs per iteration, sum of K N(N-1)/2, stay within it (an empty
     server always admits the head); it keeps enough work resident to fill the
     GPU without spreading it over every queued request, so requests finish
     close to arrival order (default 2^28; 0 = no cap) */
  uint64_t max_resident_pairs;
} trstmi_server_opts;

typedef struct trstmi_request {
  int32_t N, d;
  uint64_t seed;
  int32_t budget_iters;    /* iterations at most */
  int32_t want_phi;        /* keep the final frame for trstmi_poll */
  double target_mu;        /* stop at mu <= target_mu if > 0 ... */
  double target_rel_welch; /* ... else at mu <= target_rel_welch * Welch bound if > 0 */
  double deadline_ms;      /* 0 = none; > 0: a request not finished within deadline_ms of
                              its submission ends with TRSTMI_ETIMEOUT -- dropped from the
                              queue if it has not started, else retired at the next round
                              boundary with the iterations and mu it reached */
} trstmi_request;

typedef struct trstmi_result {
  int32_t status;          /* TRSTMI_PENDING, TRSTMI_OK or an error */
  int32_t iters;           /* iterations run */
  int32_t accepts;
  int32_t reached_target;  /* 1 if mu reached the target */
  double mu;               /* final mu (deciding precision) */
  double welch;            /* Welch bound of (N, d) */
  int64_t t_submit_ns, t_admit_ns, t_done_ns;   /* steady host clock */
  uint64_t pairs_scored;
} trstmi_result;

typedef struct trstmi_server_stats_t {
  uint64_t submitted, admitted, completed, cancelled, rounds, pairs_scored;
  double gpu_busy_s;       /* host time spent in rounds */
  size_t hbm_in_use;       /* bytes of the budget held by resident searches */
  int32_t active_slots, queued;
  int32_t worker_status;   /* TRSTMI_OK, or the error that stopped the loop */
  int32_t timed_out;       /* requests that ended with TRSTMI_ETIMEOUT */
  uint64_t kernel_launches; /* kernels the loop launched (rounds, admissions, width
                               measurements) */
} trstmi_server_stats_t;

void trstmi_default_server_opts(trstmi_server_opts *opts);
/* Starts the loop (allocates hbm_budget bytes up front). */
int trstmi_server_create(const trstmi_server_opts *opts, trstmi_server **out);
/* Stops the loop; requests still pending end as TRSTMI_ECANCELLED.  Safe on NULL. */
void trstmi_server_destroy(trstmi_server *srv);
/* Thread-safe, non-blocking.  TRSTMI_EBUSY if the queue is full. */
int trstmi_submit(trstmi_server *srv, const trstmi_request *req, uint64_t *ticket);
/* TRSTMI_PENDING while queued or running, else the request's final status;
 * out always receives what is known.  phi_out (nullable, 2*d*N doubles)
 * receives the final frame if the request asked for it. */
int trstmi_poll(trstmi_server *srv, uint64_t ticket, trstmi_result *out, double *phi_out);
/* trstmi_poll after waiting up to timeout_ms for the request to finish. */
int trstmi_wait(trstmi_server *srv, uint64_t ticket, int timeout_ms, trstmi_result *out,
                double *phi_out);
/* Cancels a queued or running request (running: at the next round boundary). */
int trstmi_cancel(trstmi_server *srv, uint64_t ticket);
int trstmi_server_stats(trstmi_server *srv, trstmi_server_stats_t *out);

/* ---------------------------------------------- scoring entry points
 * These run one stage of the iteration on the current frame without
 * changing the search state; the tests use them to compare the kernels with
 * an independent implementation on identical seeded candidates.
 */

/*
 * mu^2 of candidates c0 .. c0+count-1 of iteration t (t >= 1) drawn with
 * radius delta around the current frame, scored by the kernel of the given
 * precision: TRSTMI_FP64 (binary64 generation and Gram), TRSTMI_FP32
 * (binary32) or TRSTMI_BF16_SCREEN (the tensor-core screen alone, before
 * any re-scoring).  mu2 is a host array of count doubles.
 */
int trstmi_score(trstmi_handle h, uint32_t t, uint32_t c0, int count, double delta,
                 int precision, double *mu2);

/*
 * How the last iteration ranked its candidates (Sec. "Introduction": each
 * candidate's coherence, reduced as mu^2; the best candidate is the argmin).
 * mu2 (nullable, host, K doubles): the ranking scores of the last iteration
 * -- the binary64 mu^2 (TRSTMI_FP64), the binary32 mu^2 (TRSTMI_FP32), or in
 * the screen modes the screen's mu^2 (or the binary32 mu^2 of every
 * candidate when the iteration ranked below screen_min_delta).  Screen modes
 * only (else TRSTMI_EINVAL when requested): survivors (nullable, topk
 * indices) -- the topk smallest ranking scores, ties to the lowest index, in
 * increasing order -- and mu2_survivors (nullable, topk doubles) their
 * binary32 re-scores, from which the best (ties: lowest index) was taken.
 * Valid after trstmi_step has run at least one iteration.
 */
int trstmi_last_ranking(trstmi_handle h, double *mu2, uint32_t *survivors,
                        double *mu2_survivors);

/* Candidate c of iteration t as generated on the device in binary64
 * (precision TRSTMI_FP64) or binary32 (TRSTMI_FP32, widened), host out. */
int trstmi_candidate(trstmi_handle h, uint32_t t, uint32_t c, double delta,
                     int precision, double *out);

/*
 * mu^2 of a caller frame (host, 2*d*N doubles, columns used as given) by the
 * Gram kernel of the given precision (TRSTMI_FP64 or TRSTMI_FP32; the frame
 * is rounded to the precision first).  Stateless; device 0, default stream.
 */
int trstmi_mu2_frame(int N, int d, const double *phi, int precision, double *mu2);

/*
 * Allocation-free binary64 mu^2 of a caller frame that is already in device
 * memory.  The paper has no counterpart: this entry point exists for callers
 * that may not allocate device memory -- their device memory belongs to an
 * allocator they must not bypass (a framework's caching allocator), or they
 * run in loops where cudaMalloc / cudaFree would stall on an implicit device
 * synchronisation.  It calls no allocating routine.
 *
 * phi_dev: DEVICE pointer, 16-byte aligned, 2*d*N finite doubles in the
 *          frame layout above, columns used as given (they need not have unit
 *          norm).  mu2_dev: DEVICE pointer to one double, 8-byte aligned,
 *          written with max_{j<k} |G_jk|^2 (certified: binary32 preselection
 *          of the pairs within its rounding-error bound of the max -- the
 *          unit-column bound scaled by the largest squared column norm --,
 *          binary64 over those, a full binary64 pass if more than 65536 pairs
 *          qualify or if a squared column norm lies outside [2^-40, 2^40],
 *          where the binary32 passes could overflow or lose precision).
 * stream:  cudaStream_t to issue on (NULL = the legacy default stream).  The
 *          call only enqueues work; the result is ready when the stream is.
 * Limit:   N * d <= 131072 complex entries; larger products return
 *          TRSTMI_ESIZE without touching the device.  N < 1, d < 1, d > 256,
 *          a NULL or misaligned pointer return TRSTMI_EINVAL.
 * Scratch: one static device array of about 1.5 MiB per GPU (the binary32
 *          copy of the frame, the pair list and its counters), held by every
 *          GPU that loads the library until the process exits.  Each call
 *          clears what accumulates; the array otherwise keeps the last
 *          call's contents.  All calls share it, so calls whose work overlaps
 *          on a GPU (different streams, or different host threads) race and
 *          must be serialised by the caller.
 * The first call on a device looks up the array's device address (and sets
 * kernel attributes) for that device; make that first call before any stream
 * capture on the device.
 */
int trstmi_mu2_frame_noalloc(int N, int d, const double *phi_dev, double *mu2_dev,
                             void *stream);

/* ---------------------------------------------------------- measurement
 * The arithmetic rates that bound the library's kernels on this GPU, measured
 * by short loops that keep one unit busy on every SM (the paper has no
 * counterpart; these are the denominators of the roofline fractions the
 * benchmark reports): binary32 and binary64 fused multiply-adds (32 warps
 * per SM, eight independent chains per thread) and the tensor cores' bf16
 * and tf32 MMAs (tcgen05, M = 128, N = 256, operands in shared memory).
 * Runs on the caller's current device and the given stream (NULL = legacy
 * default stream), a few tens of milliseconds; TRSTMI_ETIMEOUT if an MMA
 * completion wait ran out (2 s).
 */
typedef struct trstmi_peaks {
  double fp32_tflops;   /* 2 flops per FFMA */
  double fp64_tflops;   /* 2 flops per DFMA */
  double tf32_tflops;   /* 2 M N K per MMA */
  double bf16_tflops;
} trstmi_peaks;

int trstmi_measure_peaks(trstmi_peaks *out, void *stream);

/* ---------------------------------------------------------- certificates
 * What a frame proves about itself (binary64, on the GPU): its coherence and
 * smallest off-diagonal |G_jk|, the lower bounds of the paper that apply to
 * its shape -- Welch (Sec. "Welch bound and equiangular lines"), orthoplex
 * and Levenshtein (for N > d^2, Proposition in Sec. "Conjectures from
 * Numerics") -- the distance of mu above the best of them, the smallest
 * chordal distance sqrt(1 - mu^2) between its lines (Sec. "Introduction"),
 * and how many distinct distances |G_jk| it has at resolution tol (the
 * single-distance observation of the same section): every |G_jk| marks bin
 * floor(|G_jk| / tol) and one distance is a maximal run of consecutive
 * marked bins, so values closer than tol always count once and values
 * farther apart than 2 tol always count twice.
 */
typedef struct trstmi_certificates {
  double mu;            /* max_{j<k} |G_jk| */
  double mu_min;        /* min_{j<k} |G_jk| */
  double welch;         /* sqrt((N-d)/(d(N-1))) for N > d, else 0 */
  double orthoplex;     /* 1/sqrt(d) for N > d^2 and d > 1, else 0 */
  double levenshtein;   /* sqrt((2N-d(d+1))/((N-d)(d+1))) for N > d^2 and d > 1, else 0 */
  double lower_bound;   /* the largest of the three */
  double gap;           /* mu - lower_bound */
  double min_chordal;   /* sqrt(1 - mu^2) */
  int32_t distinct;     /* distinct distances at resolution tol */
  int32_t reserved;
} trstmi_certificates;

/* Certificates of a host frame (2*d*N doubles, frame layout; columns are
 * normalised first).  N >= 2, 1 <= d <= 256, 1e-7 <= tol <= 1; a zero column
 * gives TRSTMI_EINVAL.  Device 0; allocates and frees device memory. */
int trstmi_frame_certificates(int N, int d, const double *phi, double tol,
                              trstmi_certificates *out);
/* Certificates of an instance's current binary64 frame (its device and
 * stream; blocks until done). */
int trstmi_instance_certificates(trstmi_handle h, double tol, trstmi_certificates *out);

/* ------------------------------------------- the paper's smooth maximum */

/*
 * The objective of the paper's optimisation procedure (Sec. "Optimization
 * procedure"): the shifted log-sum-exp
 *   F_{s,delta}(x) = s + delta * log sum_{j<k} exp((x_jk - s) / delta),
 *   x_jk = |G_jk|^2,  s = max_{j<k} x_jk,
 * of the Gram matrix G of the frame obtained by dividing each column of a
 * variable V (d x N complex) by its norm, and the real gradient of F in V.
 * By the paper's Proposition, s <= F <= s + delta log(N(N-1)/2).
 *
 * The gradient is returned as a complex array in the frame layout:
 * grad_ij = dF/dRe V_ij + i dF/dIm V_ij.  (The shift by s cancels
 * algebraically, so dF/dx_jk are the softmax weights of x / delta.)
 *
 * count frames of the same shape are evaluated together; frame q of v is
 * the 2*d*N doubles at v + 2*d*N*q.  precision: TRSTMI_FP64 (binary64
 * throughout) or TRSTMI_FP32 (the variable rounded to binary32, Gram,
 * weights, block products and each column's sum over its tiles in binary32;
 * S, F and the projection through the normalisation in binary64).  Requires N >= 2, 1 <= d <= 256,
 * count >= 1, 0 < delta < inf, count*N*d < 2^31; a zero column makes that
 * frame's results NaN (TRSTMI_EINVAL from trstmi_lse_frames).  The results
 * do not depend on the order in which the device runs its tiles.
 */

/* Host buffers (v: count*2*d*N doubles; F, s (nullable): count doubles;
 * grad (nullable): count*2*d*N doubles).  Device 0, default stream;
 * allocates and frees its device memory, blocks until done. */
int trstmi_lse_frames(int N, int d, int count, const double *v, double delta, int precision,
                      double *F, double *s, double *grad);

/* Bytes of device scratch that trstmi_lse_frames_device needs. */
int trstmi_lse_scratch_bytes(int N, int d, int count, int precision, size_t *bytes);

/*
 * Allocation-free form on device buffers of the current device: v_dev
 * (count*2*d*N doubles), scratch_dev (256-byte aligned, at least
 * trstmi_lse_scratch_bytes), out_dev (count x [F, s] doubles), grad_dev
 * (count*2*d*N doubles, or NULL for the value alone).  Only enqueues work on
 * `stream` (NULL = legacy default stream); the results are ready when the
 * stream is.  Calls sharing one scratch array must not overlap.
 */
int trstmi_lse_frames_device(int N, int d, int count, const double *v_dev, double delta,
                             int precision, void *scratch_dev, size_t scratch_bytes,
                             double *out_dev, double *grad_dev, void *stream);

/* ------------------------------------ trust-region CG-Steihaug procedure
 * The paper's optimisation procedure on one frame (Sec. "Optimization
 * procedure"; Algorithm "TRSTMI optimization steps", step 2): for each
 * smoothing parameter delta_k in turn (a decreasing sequence), trust-region
 * iterations on F_{s,delta_k} over the variable V, each step from CG-Steihaug
 * (Algorithm "Trust-Region CG-Steihaug", after Nocedal and Wright Alg. 7.2),
 * the result of one stage starting the next.  Per iteration (Nocedal and
 * Wright Alg. 4.1): g = grad F; the stage ends when |g| <= gtol or after
 * max_outer iterations or when the radius falls below 1e-14; the step p
 * solves the model with CG tolerance eps = min(1/2, sqrt|g|) |g| and at most
 * max_cg iterations; rho = (F(V) - F(V + p)) / (m(0) - m(p)); the radius is
 * divided by 4 if rho < 1/4 and doubled (up to radius_max) if rho > 3/4 and
 * the step reached it; the step is taken if rho > eta, after which each
 * column of V is divided by its norm (F does not change).  The radius starts
 * at radius0 in every stage.  The model's B is the Hessian of F at the
 * iterate, as in the paper's Algorithm (B_k = grad^2 f_k): its products are
 * formed exactly, by differentiating the gradient along the direction (the
 * chain rule through the normalisation, the Gram entries and the softmax
 * weights); hessian = 1 selects central differences of the gradient (step
 * fd_step) instead, a diagnosis option.  Binary64 throughout, on the GPU
 * (F, its gradient and the Hessian products by device kernels, every vector
 * operation and inner product in device kernels; the host keeps the
 * scalars, or, on the resident path, one CTA runs the whole procedure).
 */
typedef struct trstmi_tr_options {
  int32_t n_delta;      /* stages, 1..16 */
  int32_t max_outer;    /* trust-region iterations per stage (default 100) */
  double delta[16];     /* smoothing parameters (default 0.1, 0.03, 0.01, 0.003, 0.001,
                           3e-4, 1e-4), each > 0 */
  int32_t max_cg;       /* CG iterations per step (default 200), >= 1 */
  int32_t path;         /* 0 (default): frames that fit in one CTA's shared memory (up
                           to about d = 9, N = 81) run resident, one CTA per frame,
                           larger ones as a stack driven from the host; 1: always the
                           stack; 2: always resident (TRSTMI_EUNSUPPORTED if a frame
                           does not fit).  Both run the same algorithm; their sums
                           are ordered differently. */
  double radius0;       /* initial radius of every stage (default 0.1), > 0 */
  double radius_max;    /* radius cap (default 1.0), >= radius0 */
  double eta;           /* acceptance threshold on rho (default 1e-4), in [0, 1/4) */
  double gtol;          /* stage ends when |grad F| <= gtol (default 1e-9), >= 0 */
  double fd_step;       /* difference step of hessian = 1 (default 1e-6), > 0 */
  int32_t hessian;      /* 0 (default): exact Hessian products; 1: central differences */
  int32_t reserved;
} trstmi_tr_options;

/* One row per trust-region iteration. */
typedef struct trstmi_tr_row {
  int32_t stage, iter;
  double F;             /* F_{s,delta} at the iterate */
  double s;             /* max |G_jk|^2 at the iterate */
  double gnorm;         /* |grad F| */
  double radius;        /* radius the step was solved in */
  double rho;           /* actual / predicted decrease (-1 if the prediction was not positive) */
  double step_norm;     /* |p| */
  double pred;          /* m(0) - m(p) */
  int32_t cg_iters;     /* CG iterations of the step */
  int32_t cg_status;    /* 0 residual below eps, 1 boundary, 2 negative curvature, 3 limit */
  int32_t accepted;
  int32_t reserved;
} trstmi_tr_row;

/* Fills *o with the defaults listed above. */
void trstmi_tr_default_options(trstmi_tr_options *o);

/* The procedure on a host frame phi (2*d*N doubles, frame layout), replaced
 * by the result (unit columns).  trace (nullable): up to cap rows; *n_rows
 * (nullable): rows produced.  N >= 2, 1 <= d <= 256; a zero column gives
 * TRSTMI_EINVAL.  Device 0; allocates and frees its device memory. */
int trstmi_tr_solve(int N, int d, double *phi, const trstmi_tr_options *o,
                    trstmi_tr_row *trace, int cap, int *n_rows);

/* The paper's whole algorithm (Algorithm "TRSTMI optimization steps"): L
 * random initialisations -- trial i starts from the frame trstmi_create
 * draws for seed seed0 + i -- each run through the procedure above, and the
 * minimum over the trials.  The trials advance together as one stack of
 * frames on the GPU, at most batch_cap at a time (<= 0: all), and each
 * follows exactly the trajectory trstmi_tr_solve gives it alone.  L <= 0
 * selects 2 d^2 trials.  out: the minimum of mu over the trials (binary64),
 * its trial (lowest index on ties) and seed.  mu_all (nullable): L doubles.
 * best_phi (nullable): 2*d*N doubles, the winning frame.  trace (nullable):
 * up to cap rows of the winning trial; *n_rows (nullable) its row count.
 * work (nullable, host): 2*L ints, for trial i its trust-region iterations
 * (work[2i], the rows it would trace) and Hessian-vector products
 * (work[2i+1]); each iteration evaluates F and its gradient once and F once
 * more at the trial point, each product two gradients. */
int trstmi_tr_multistart(int N, int d, uint64_t seed0, int L, const trstmi_tr_options *o,
                         int batch_cap, trstmi_multistart_result *out, double *mu_all,
                         double *best_phi, trstmi_tr_row *trace, int cap, int *n_rows,
                         int *work);

/* The procedure applied to an instance's current frame (polishing a
 * search's result), on the instance's device: the frame is replaced by the
 * procedure's result and recertified, as with trstmi_set_phi. */
int trstmi_instance_tr_solve(trstmi_handle h, const trstmi_tr_options *o,
                             trstmi_tr_row *trace, int cap, int *n_rows);

/* ------------------------------------------------- measurement entry point */

/*
 * Times the candidate-scoring kernel of the instance alone: `launches`
 * launches over the instance's K candidates (iteration t = 1, 2, ...; radius
 * delta around the current frame), each bracketed by CUDA events on the
 * instance's stream.  Between launches, outside the timed spans, flush_bytes
 * of device scratch (0 = none) are overwritten so each launch starts with a
 * cold L2.  *avg_ms receives the mean device time of one launch.  The
 * precision selects the kernel: TRSTMI_FP64 / TRSTMI_FP32 (SIMT Gram) or
 * TRSTMI_BF16_SCREEN (tensor-core screen).  Does not change the search state.
 */
int trstmi_profile_score(trstmi_handle h, int precision, int launches, double delta,
                         size_t flush_bytes, double *avg_ms);

/*
 * Exercises the bounded device-side waits; the paper has no counterpart.
 * Every wait inside the tensor-core screen (a consumer waiting for a column
 * block, the MMA issuer waiting for a free accumulator, the epilogue waiting
 * for a finished tile) gives up after a time limit instead of spinning
 * forever, flags TRSTMI_ETIMEOUT and lets the other roles of the CTA leave,
 * so a stalled launch ends and the CUDA context stays usable.  This call
 * launches the screen of the given precision (TRSTMI_BF16_SCREEN,
 * TRSTMI_FP16_SCREEN or TRSTMI_TF32_SCREEN) over min(K, 8) candidates of the
 * instance with its block producers withheld, so the first wait can never
 * complete, and with the limit shortened to wait_limit_ms (0 < limit <=
 * 2000; the screen's normal limit is 2000 ms).  Blocks until the launch
 * ends.  Returns TRSTMI_ETIMEOUT when the wait ran out as intended,
 * TRSTMI_OK if it did not, TRSTMI_EUNSUPPORTED outside the screen's range
 * and TRSTMI_EINVAL on bad arguments.  Uses only the instance's scoring
 * scratch; the search state is unchanged.
 */
int trstmi_screen_wait_test(trstmi_handle h, int precision, double wait_limit_ms);

#ifdef __cplusplus
}
#endif
#endif /* TRSTMI_H */
