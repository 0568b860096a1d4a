/*
 * hs.h -- C ABI of the GB300-native batched SPHINCS+ signer (libhs.so).
 *
 * Scheme: SPHINCS+ round 3.1, SHA2 "simple" instantiation, at the -f
 * parameter sets of Table 1 of HERO-Sign (arxiv 2512.23969):
 *   128f (n=16, h=66, d=22, h'=3, a=6, k=33)  17088-byte signatures
 *   192f (n=24, h=66, d=22, h'=3, a=8, k=33)  35664-byte signatures
 *   256f (n=32, h=68, d=17, h'=4, a=9, k=35)  49856-byte signatures
 * F and PRF use SHA-256; H, T_l, H_msg and PRF_msg use SHA-256 at n=16 and
 * SHA-512 at n=24/32.  Signing is deterministic (opt_rand = PK.seed).
 * Signing follows the paper's decomposition (Sec. III, Fig. 2): a message
 * stage (R and digest), FORS_Sign (Sec. III-B), TREE_Sign (Sec. III-A) and
 * WOTS+_Sign, all as sm_103a kernels; nothing runs on the CPU.
 *
 * Conventions shared by every call:
 *  - Byte strings are packed, unpadded uint8_t arrays.  Keys, messages and
 *    signatures are laid out contiguously in index order.
 *  - Every buffer is owned by the caller and must stay valid until the work
 *    enqueued on 'stream' has completed.  The library keeps no pointer
 *    after a call returns.
 *  - 'stream' is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls whose buffers are all device memory are asynchronous:
 *    they enqueue kernels on 'stream' and return HS_OK once the launches
 *    succeeded.  If any input or output buffer is host memory (pageable or
 *    pinned), the call stages it through device memory and synchronizes
 *    'stream' before returning, so host outputs are ready on return.
 *  - Argument errors are detected on the host and returned synchronously;
 *    nothing is enqueued in that case.  Errors found by the kernels (a key
 *    index out of range) are OR-ed into a per-device status word that
 *    hs_check_status() reads.  No call traps, asserts or aborts.
 *  - count == 0 is a valid no-op.
 *  - Scratch memory is taken from the device's stream-ordered memory pool
 *    (cudaMallocAsync on 'stream') and returned to it on the same stream.
 */
#ifndef HS_H_
#define HS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Parameter sets.  HS_128F/192F/256F are the sets the paper signs with
 * (its Table 1).  HS_TOY is a test-only miniature (n=16, h=4, d=2, h'=2,
 * a=3, k=4, 1456-byte signatures) with no security; it exists so that every
 * tree of the hypertree can be brute-forced in tests.  HS_128S/192S/256S are
 * the scheme's small-signature sets (a variant the paper does not use):
 * (n, h, d, h', a, k) = (16, 63, 7, 9, 12, 14), (24, 63, 7, 9, 14, 17),
 * (32, 64, 8, 8, 14, 22); 7856 / 16224 / 29792-byte signatures.
 * HS_SHAKE_* are the SHAKE256 instantiations of the six sets (SPHINCS+ SHAKE-simple, FIPS 205
 * Sec. 11.1): same sizes and key layout, every hash SHAKE256 with the full
 * 32-byte address; another variant the paper does not use.
 * HS_ROBUST_* are the robust SHA2 instantiations of the three f sets
 * (SPHINCS+ round 3.1 SHA2-robust): F, H and T_l hash their input xor
 * MGF1-SHA-x(PK.seed || ADRSc, input length), SHA-x being the hash the
 * tweakable hash itself uses; PRF, PRF_msg and H_msg as in the simple sets.
 * Same sizes and key layout; keys and signatures differ from the simple
 * sets'.  A variant the paper does not use; FIPS 205 has no robust sets, so
 * the hs_slh_* calls refuse them. */
typedef enum {
    HS_128F = 0, HS_192F = 1, HS_256F = 2, HS_TOY = 3,
    HS_128S = 4, HS_192S = 5, HS_256S = 6,
    HS_SHAKE_128F = 7, HS_SHAKE_192F = 8, HS_SHAKE_256F = 9,
    HS_SHAKE_128S = 10, HS_SHAKE_192S = 11, HS_SHAKE_256S = 12,
    HS_ROBUST_128F = 13, HS_ROBUST_192F = 14, HS_ROBUST_256F = 15
} hs_params;
#define HS_NUM_PARAMS 16

typedef enum {
    HS_OK = 0,
    HS_EINVAL = 1,   /* bad enum, NULL pointer, size overflow, mixed buffer kinds */
    HS_ENOMEM = 2,   /* device memory for scratch or staging could not be obtained */
    HS_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
    HS_ETIMEOUT = 4, /* a bounded wait ran out */
    HS_EKEY = 5,     /* a key index was >= the number of keys */
    HS_ECANCELED = 6,/* a server request was cancelled before it ran */
    HS_EBUDGET = 7   /* a server request can never fit the server's memory budget */
} hs_status;

/* Sizes in bytes for a parameter set; 0 for an invalid enum.
 * seed = SK.seed || SK.prf || PK.seed (3n); pk = PK.seed || PK.root (2n);
 * sk = SK.seed || SK.prf || PK.seed || PK.root (4n). */
size_t hs_sig_bytes(hs_params p);
size_t hs_pk_bytes(hs_params p);
size_t hs_sk_bytes(hs_params p);
size_t hs_seed_bytes(hs_params p);

/*
 * hs_keygen -- derive 'count' key pairs from 'count' seeds.
 * Definition: PK.root is the root of the single XMSS tree of the top
 * hypertree layer d-1 (tree 0), built from WOTS+ public keys (Sec. II-A-3/4).
 *   seeds : count x 3n bytes (SK.seed || SK.prf || PK.seed), host or device
 *   pk    : count x 2n bytes out, host or device
 *   sk    : count x 4n bytes out, host or device
 * Errors: HS_EINVAL for a bad enum or a NULL pointer with count > 0.
 */
hs_status hs_keygen(hs_params p, const uint8_t *seeds, uint32_t count,
                    uint8_t *pk, uint8_t *sk, void *stream);

/*
 * hs_sign_batch -- sign 'count' messages (paper Fig. 2 per message:
 * hash_message, message_to_indices, fors_sign, d x merkle_sign).
 *   sk      : num_keys x 4n bytes (hs_keygen's sk layout)
 *   key_idx : count x uint32, key of each message; NULL = key 0 for all
 *   msgs    : all messages concatenated in order (sum(lens) bytes; may be
 *             NULL when every length is 0)
 *   lens    : count x uint64 message lengths in bytes
 *   sigs    : count x hs_sig_bytes(p) bytes out; signature i at i*SIG
 * Message i starts at the sum of lens[0..i-1]; the offsets are computed on
 * the device.  If msgs is host memory, lens must be host memory too (its
 * total sizes the staging copy).
 * Errors: HS_EINVAL (bad enum, NULL sk/lens/sigs with count > 0,
 * num_keys == 0), HS_ENOMEM, HS_ECUDA.  A key_idx entry >= num_keys sets
 * HS_EKEY in the status word; that message's signature bytes are zero.
 */
hs_status hs_sign_batch(hs_params p, const uint8_t *sk, uint32_t num_keys,
                        const uint32_t *key_idx, const uint8_t *msgs,
                        const uint64_t *lens, uint32_t count, uint8_t *sigs,
                        void *stream);

/*
 * hs_sign_mixed -- several signing jobs, possibly under different parameter
 * sets, in one call (the paper's batched form, Sec. III-F: per batch a DAG
 * of {FORS_Sign || TREE_Sign} -> WOTS+_Sign; here every job's DAG runs on
 * its own pair of streams, all forked from and joined into 'stream').
 *   jobs[j] : one hs_sign_batch worth of arguments; device buffers only
 *   njobs   : 0..16 (jobs with count 0 are skipped)
 *   use_graph: 1 = the whole fork/join sequence is captured into one CUDA
 *             graph and launched once; 0 = the same launches go out directly
 * Asynchronous on 'stream'; signatures are identical to hs_sign_batch's.
 * The graph form keeps its graph and its scratch (a device buffer the
 * library owns, grown as needed and kept until the process exits) from
 * call to call: a call with the same jobs (same buffers, counts and sets)
 * and the same tuning relaunches the graph without capturing it again; a
 * call of the same shape updates it in place.  Graph-form calls on a
 * device share that buffer, so each waits on the GPU for the previous one.
 * Errors: HS_EINVAL (bad set, NULL or host buffer, more than 16 jobs),
 * HS_ENOMEM, HS_ECUDA.  Key-index errors go to the status word.
 * Calls must not be issued concurrently from several host threads.
 */
typedef struct {
    hs_params params;
    const uint8_t *sk;
    uint32_t num_keys;
    const uint32_t *key_idx;
    const uint8_t *msgs;
    const uint64_t *lens;
    uint32_t count;
    uint8_t *sigs;
} hs_sign_job;
hs_status hs_sign_mixed(const hs_sign_job *jobs, uint32_t njobs, int use_graph, void *stream);

/*
 * hs_verify_batch -- verify 'count' signatures (the scheme's verification:
 * FORS public key from the FORS signature, then d WOTS+ public keys from
 * their signatures and auth-path climbs, compared with PK.root).
 *   pk      : num_keys x 2n bytes (PK.seed || PK.root)
 *   key_idx : count x uint32 or NULL (key 0)
 *   msgs, lens : as in hs_sign_batch
 *   sigs    : count x hs_sig_bytes(p)
 *   ok      : count bytes out; 1 = valid, 0 = invalid (not an error)
 * Errors: as hs_sign_batch; an out-of-range key gives ok = 0 and HS_EKEY.
 */
hs_status hs_verify_batch(hs_params p, const uint8_t *pk, uint32_t num_keys,
                          const uint32_t *key_idx, const uint8_t *msgs,
                          const uint64_t *lens, const uint8_t *sigs,
                          uint32_t count, uint8_t *ok, void *stream);

/*
 * hs_check_status -- synchronize 'stream', then return and clear the status
 * word of the current device (an OR of (1u << hs_status) bits raised by
 * kernels since the last check).  *flags may be NULL.
 */
hs_status hs_check_status(void *stream, uint32_t *flags);

/* Text of the most recent error of the calling thread: argument and launch
 * errors found on the host, and the key-index error hs_check_status reports
 * for the kernels.  The text stays until the thread's next error (calls that
 * succeed do not clear it).  hs_last_error returns a pointer that stays
 * valid until that next error; hs_last_error_copy copies the text into the
 * caller's buffer of 'len' bytes, truncated to len - 1 bytes and always
 * NUL-terminated, and returns HS_EINVAL (copying nothing) if buf is NULL or
 * len is 0. */
const char *hs_last_error(void);
hs_status hs_last_error_copy(char *buf, size_t len);

/*
 * Per-stage timing for measurement.  While enabled, every hs_sign_batch call
 * records CUDA events around each of its kernels on its own stream.
 * hs_profile_read synchronizes those events and writes, for the most recent
 * call, up to 'max' stage durations in milliseconds into ms[] and their
 * names (static strings) into names[] (either may be NULL); it returns the
 * number of stages, or -1 if no profiled call has happened.
 * Stages: 0 keyprep, 1 offsets, 2 message, 3 fors, 4 fors_pk, 5 tree, 6 wots.
 */
void hs_profile_enable(int on);
int hs_profile_read(float *ms, const char **names, int max);

/*
 * hs_probe_int_pipes -- measure the current GPU's integer issue rates for the
 * roofline (the signer does not depend on it).  Writes up to 'max' rates in
 * lane-operations per clock per SM, from SM cycle counters, for: 0 LOP3,
 * 1 SHF (funnel shift), 2 IADD, 3 IMAD, 4 IMAD.HI, 5 PRMT, 6 LOP3+IMAD
 * interleaved.  Synchronizes the device and allocates a few KB temporarily.
 * Returns the number of rates written, or -1 on a CUDA error.
 */
int hs_probe_int_pipes(float *rates, int max);

/*
 * hs_probe_sha_mix -- measure the ceiling of the SHA-2 instruction mix
 * itself on the current GPU, for the roofline's "SHA-mix peak" (the scheme's
 * work is SHA-256 / SHA-512 compressions, FIPS 180-4 Sec. 6.2 / 6.4, and the
 * signer does not depend on this call).  The signer's own compression
 * functions run back to back on an independent state per thread, one wave
 * of full-occupancy blocks, timed by SM cycle counters.  Writes up to 'max'
 * rates: 0 SHA-256 compressions per clock per SM (all 64 rounds, with the
 * signer's round code: additions on the FMA pipe), 1 SHA-512 compressions
 * per clock per SM (80 rounds on 32-bit halves), 2 64-bit additions (two
 * 32-bit halves and a carry) in lane-operations per clock per SM, 3 SHA-256
 * compressions per clock per SM as FIPS 180-4 writes them (every addition
 * left to the compiler).  Synchronizes the device and allocates a few KB
 * temporarily.
 * Returns the number of rates written, or -1 on a CUDA error.
 */
int hs_probe_sha_mix(float *rates, int max);

/* Number of kernels one hs_sign_batch call launches (for launch accounting). */
int hs_sign_kernel_count(void);

/*
 * hs_set_chain_checkpoint -- process-wide tuning knob of hs_sign_batch.
 * TREE_Sign computes every chain of every WOTS+ key pair of the hypertree,
 * including the signing key pair whose chains WOTS+_Sign needs again at the
 * message digits (Sec. III: WOTS+_Sign runs after TREE_Sign).  With a stride
 * s in {1, 2, 4, 8}, TREE_Sign stores every s-th position of the signing key
 * pair's chains in scratch (count * d * len * (16 / s) * n bytes; 1.6 GB for
 * 16384 128f signatures at s = 2) and WOTS+_Sign finishes each chain in fewer
 * than s steps; s = 0 stores nothing and WOTS+_Sign recomputes each chain
 * from its secret.  Signatures are identical for every setting.  Default 2.
 * This sets the stride of every parameter set (hs_tune_set with
 * HS_TUNE_CHECKPOINT then sets one set's own).  Returns HS_EINVAL for any
 * other value.  Not thread-safe against concurrent signing calls.
 */
hs_status hs_set_chain_checkpoint(uint32_t stride);

/*
 * Launch-shape tuning, per parameter set (process-wide).  Signatures are
 * identical for every setting; only speed changes.  Knobs:
 *   HS_TUNE_FORS_LANES      lanes of a warp that share one FORS tree
 *                           (each lane builds a subtree of 2^a / lanes
 *                           leaves, the rest merges by shuffles); a batch
 *                           too small to give FORS_Sign about 1024 threads
 *                           per SM takes the next wider compiled value
 *   HS_TUNE_TREE_MIN_BLOCKS minimum resident 128-thread blocks per SM that
 *                           TREE_Sign is compiled for (0 = compiler's choice)
 *   HS_TUNE_TREE_SPLIT_BELOW batches of fewer messages than this run
 *                           TREE_Sign chain-parallel (a thread per WOTS+
 *                           chain, then a thread per leaf for T_len and the
 *                           Merkle levels); 0 = never.  Any value >= 0 is
 *                           accepted; hs_tune_options lists suggestions.
 *                           Extra scratch: len * n bytes per hypertree leaf.
 *   HS_TUNE_TREE_POLICY     where TREE_Sign's SHA-256 additions run: 7 =
 *                           round additions on the FMA pipe (IMAD), 15 =
 *                           the message-schedule sums too (SHA-2 sets)
 *   HS_TUNE_TREE_CHAINS     WOTS+ chains a TREE_Sign thread runs at once:
 *                           1, or 2 interleaved (more independent work per
 *                           thread, more registers; SHA-2 sets)
 *   HS_TUNE_CHECKPOINT      this set's chain checkpoint stride (0, 1, 2, 4,
 *                           8; see hs_set_chain_checkpoint, which sets every
 *                           set's stride at once)
 *   HS_TUNE_TREE_STEP_US,   measured costs of the two TREE_Sign forms (0 =
 *   HS_TUNE_TREE_SPLIT_NS   not measured): the per-leaf form's time for one
 *                           warp per SM sub-partition, in us, and the
 *                           chain-parallel form's time per message, in ns.
 *                           At or above HS_TUNE_TREE_SPLIT_BELOW, a batch
 *                           within four such per-leaf steps takes the form
 *                           they predict faster (the per-leaf time grows in
 *                           whole steps); any value >= 0 is accepted
 *   HS_TUNE_MSG_WARP_BELOW  batches of fewer messages than this hash each
 *                           message (PRF_msg, H_msg; Sec. II-A) with a whole
 *                           warp: the message schedules of up to 32 blocks
 *                           are computed at once, one block per lane, so a
 *                           long message's serial hash runs only its rounds
 *                           (SHA-2 sets; the SHAKE sets accept 0 only);
 *                           0 = always a thread per message; any value >= 0
 *                           is accepted.  The server (hs_server_*) takes this
 *                           form only for a batch with no other batch of
 *                           its own in flight
 * TREE_Sign's per-leaf kernel is compiled for its default combination of
 * min blocks, policy and chains per thread, and for each alternative value
 * of one knob with the other two at their defaults (min blocks 0, the
 * set's default policy, 1 chain); other combinations are refused.
 * hs_tune_options lists the compiled values (returns their number, or -1);
 * hs_tune_set returns HS_EINVAL for a value, or a TREE_Sign combination,
 * that is not compiled in; hs_tune_get returns the current value (-1 for
 * bad arguments).  The package's autotuner measures these and stores the
 * best per device.
 */
typedef enum {
    HS_TUNE_FORS_LANES = 0, HS_TUNE_TREE_MIN_BLOCKS = 1, HS_TUNE_TREE_SPLIT_BELOW = 2,
    HS_TUNE_TREE_POLICY = 3, HS_TUNE_TREE_CHAINS = 4, HS_TUNE_CHECKPOINT = 5,
    HS_TUNE_TREE_STEP_US = 6, HS_TUNE_TREE_SPLIT_NS = 7, HS_TUNE_MSG_WARP_BELOW = 8
} hs_tune_knob;
int hs_tune_options(hs_params p, int knob, int32_t *values, int max);
hs_status hs_tune_set(hs_params p, int knob, int32_t value);
int32_t hs_tune_get(hs_params p, int knob);

/*
 * Continuous-batching signing server.  Requests (parameter set, key index,
 * message) are submitted at any time; a scheduler thread keeps up to
 * max_inflight batches on the GPU, each on its own stream, and launches the
 * next batch -- the oldest pending requests of one parameter set, at most
 * max_batch of them and at most max(256, all pending / max_inflight), so a
 * backlog near capacity is spread over the slots rather than formed into
 * one long batch -- as soon as a slot and memory are free, so newly
 * arrived requests overlap with running ones.  Device memory for messages,
 * signatures and scratch comes from one arena of mem_budget_bytes reserved
 * at creation (admission control: a batch that does not fit waits); host
 * staging uses a pinned arena of pinned_bytes (0 = half the budget).  Keys
 * and their SHA-2 midstates are resident on the device from creation.
 * Signatures equal hs_sign_batch's for the same key and message.
 *
 * hs_server_create: sks[p] = nkeys[p] keys of set p (4n bytes each, host or
 *   device; nkeys[p] = 0 disables set p).  The current device is used.
 * hs_server_submit: copies the message; the signature is written to sig_out
 *   (host memory, hs_sig_bytes(p) bytes, valid until completion; NULL =
 *   compute and discard, for load tests).  HS_EKEY for a key index >= nkeys;
 *   HS_EBUDGET for a request that alone needs more device or pinned memory
 *   than the server reserved (it could never be admitted); HS_EINVAL for
 *   malformed arguments (NULL server, bad set, NULL message of nonzero
 *   length).
 * hs_server_wait: blocks up to timeout_ms; HS_ETIMEOUT if still pending.
 * hs_server_poll: hands out each finished request once (id, latency from
 *   arrival to host-observed completion in ns, and its hs_status: HS_OK,
 *   HS_ECUDA for a failed batch, HS_ECANCELED) and forgets it.  Any of the
 *   three output arrays may be NULL.
 * hs_server_replay: open-loop load generator: submits request i (set
 *   params[i], key keys[i], message pool entry pool_idx[i] of the packed pool
 *   pool_msgs / pool_lens) at arrival_ns[i] after the call starts, waits for
 *   all, and reports each latency from its scheduled arrival.  Signatures go
 *   to sigs + sig_offsets[i], or are discarded if sigs is NULL.
 *   HS_ETIMEOUT after timeout_ms; HS_ECUDA if any request's batch failed.
 * hs_server_destroy: stops the scheduler, waits for running batches, frees
 *   everything; requests never launched are dropped.
 * With cache_layers > 0 each served set keeps its keys as a keyset with
 *   that many top layers prebuilt (capped at d - 1; see hs_keyset_create
 *   for the device memory it takes, outside mem_budget_bytes).
 * Failures: a batch whose launch fails completes all its requests with
 *   HS_ECUDA (counted in stats.failed).  A real CUDA error also makes the
 *   server's status (hs_server_get_stats' return) HS_ECUDA; later batches
 *   are still attempted, and the caller decides whether to recreate it.
 */
typedef struct hs_server hs_server;
typedef struct {
    uint32_t max_inflight;      /* batches on the GPU at once (1..16) */
    uint32_t max_batch;         /* requests per batch */
    uint64_t mem_budget_bytes;  /* device arena for in-flight work (>= 1 MiB) */
    uint64_t pinned_bytes;      /* pinned host staging arena (0 = budget / 2) */
    uint32_t cache_layers;      /* top hypertree layers prebuilt per key (hs_keyset; 0 = none) */
} hs_server_config;
typedef struct {
    uint64_t completed, batches, batched_requests, pending;
    uint64_t max_device_bytes_in_use;
    uint32_t max_inflight_batches;
    uint64_t failed;            /* requests completed with HS_ECUDA */
    uint64_t cancelled;         /* requests completed with HS_ECANCELED */
} hs_server_stats;
hs_status hs_server_create(const hs_server_config *cfg, const uint8_t *const sks[HS_NUM_PARAMS],
                           const uint32_t nkeys[HS_NUM_PARAMS], hs_server **out);
hs_status hs_server_submit(hs_server *s, hs_params p, uint32_t key, const uint8_t *msg,
                           uint64_t len, uint8_t *sig_out, uint64_t *id);
hs_status hs_server_wait(hs_server *s, uint64_t id, uint32_t timeout_ms);
int hs_server_poll(hs_server *s, uint64_t *ids, uint64_t *latency_ns, int32_t *status, int max);
hs_status hs_server_get_stats(hs_server *s, hs_server_stats *st);
hs_status hs_server_replay(hs_server *s, uint32_t count, const uint8_t *params,
                           const uint32_t *keys, const uint32_t *pool_idx,
                           const uint8_t *pool_msgs, const uint64_t *pool_lens,
                           uint32_t pool_count, const uint64_t *arrival_ns, uint8_t *sigs,
                           const uint64_t *sig_offsets, uint64_t *latency_ns,
                           uint32_t timeout_ms);
hs_status hs_server_destroy(hs_server *s);

/*
 * hs_server_cancel: drops a request that is still waiting for a batch; its
 * wait then returns HS_ECANCELED and poll reports it.  HS_EINVAL if the id
 * is unknown, already running or finished (a running batch always completes).
 * hs_server_inject_launch_failures: test hook -- the next n batches the
 * scheduler forms are treated as if their launch had failed (nothing is
 * launched; their requests complete with HS_ECUDA) so that callers can test
 * how they handle a failed batch without faulting a GPU.
 */
hs_status hs_server_cancel(hs_server *s, uint64_t id);
hs_status hs_server_inject_launch_failures(hs_server *s, uint32_t n);

/*
 * hs_set_tree_sharing -- process-wide switch (default off) for hs_sign_batch
 * and hs_sign_mixed.  The XMSS tree a message signs with at layer j depends
 * only on (key, j, idx_tree >> (j h')) (paper Fig. 2), so in a batch where
 * many messages share a key the upper layers repeat the same trees.  When
 * on, each batch finds its distinct trees in the layers where at most half
 * as many distinct trees as messages are possible, builds each of them once
 * and copies every message's auth path and root from it.  Signatures are
 * byte-identical either way; only repeated work is skipped (about 16 % of
 * TREE_Sign for 16384 messages over 16 keys).  Extra scratch per distinct
 * shared tree: its nodes and the checkpoints of all its leaves.
 */
hs_status hs_set_tree_sharing(int on);

/*
 * hs_set_host_direct -- process-wide switch (default on) for signing calls
 * whose signature buffer is page-locked host memory mapped into the device
 * address space (cudaHostAlloc / cudaMallocHost; every such buffer is mapped
 * under unified addressing): the kernels then write the signatures into it
 * directly (on GB300 over the coherent NVLink-C2C link) instead of into a
 * device staging buffer followed by a device-to-host copy.  The call still
 * returns after the signatures are complete.  Off: always stage and copy.
 * Other host memory is always staged.
 */
hs_status hs_set_host_direct(int on);

/*
 * FIPS 205 (SLH-DSA) mode -- a variant; the paper signs with SPHINCS+
 * round 3.1.  At every set here (SHA2 and SHAKE) FIPS 205 keeps the keys,
 * tweakable hashes, addresses and sizes and changes two things: the FORS
 * indices are the base-2^a digits of md read most significant bit first
 * (base_2b), and pure signing signs M' = 0x00 || len(ctx) || ctx || M.
 * hs_slh_sign_batch / hs_slh_verify_batch are SLH-DSA.Sign (deterministic:
 * opt_rand = PK.seed) and SLH-DSA.Verify for a batch, with one context
 * string ctx (host memory, ctx_len <= 255) for the whole call; ctx_len =
 * HS_SLH_INTERNAL signs / verifies the messages as given (FIPS 205's
 * internal functions).  Keys come from hs_keygen.  Other arguments, layouts
 * and errors as hs_sign_batch / hs_verify_batch; HS_EINVAL for ctx_len 256
 * .. 0xFFFFFFFE.
 */
#define HS_SLH_INTERNAL 0xFFFFFFFFu
hs_status hs_slh_sign_batch(hs_params p, const uint8_t *sk, uint32_t num_keys, const uint32_t *key_idx,
                            const uint8_t *ctx, uint32_t ctx_len, const uint8_t *msgs,
                            const uint64_t *lens, uint32_t count, uint8_t *sigs, void *stream);
hs_status hs_slh_verify_batch(hs_params p, const uint8_t *pk, uint32_t num_keys,
                              const uint32_t *key_idx, const uint8_t *ctx, uint32_t ctx_len,
                              const uint8_t *msgs, const uint64_t *lens, const uint8_t *sigs,
                              uint32_t count, uint8_t *ok, void *stream);

/*
 * Keysets: signing keys kept resident on the device with the top hypertree
 * layers prebuilt.  For a key, the tree of layer j a message signs with is
 * fixed by idx_tree >> (j h') (paper Fig. 2), which takes 2^((d-1-j) h')
 * values; a keyset builds all of them once for its top cache_layers layers
 * (j = d - cache_layers .. d-1), with every Merkle node and the WOTS+ chain
 * checkpoints of every leaf, so each later signature builds only its lower
 * d - cache_layers layers and copies the rest.  Signatures are
 * byte-identical to hs_sign_batch's with the same keys.
 *
 * hs_keyset_create: sk = num_keys keys (4n bytes each, host or device; the
 *   keyset keeps its own copy); cache_layers in 0..d-1 (0 = resident keys
 *   only), at most 2^24 trees per key and 2^32 in all.  The chain
 *   checkpoint stride in force (hs_set_chain_checkpoint) is fixed into the
 *   keyset.  Enqueued on 'stream' and waited for before returning; the
 *   keyset belongs to the current device.  HS_ENOMEM if it does not fit.
 *   Cached trees per key: sum over u < cache_layers of 2^(u h'); device
 *   bytes per tree: 2^h' (2 n + len n 16 / stride) (about 36 KB at 128f,
 *   stride 2) -- hs_keyset_bytes gives the total.
 * hs_sign_keyset: as hs_sign_batch with the keyset's keys (key_idx indexes
 *   them; NULL = key 0); call it on the keyset's device.
 * hs_keyset_destroy: frees it (waits for the device); NULL is a no-op.
 */
typedef struct hs_keyset hs_keyset;
hs_status hs_keyset_create(hs_params p, const uint8_t *sk, uint32_t num_keys, uint32_t cache_layers,
                           void *stream, hs_keyset **out);
size_t hs_keyset_bytes(const hs_keyset *ks);
hs_status hs_sign_keyset(const hs_keyset *ks, const uint32_t *key_idx, const uint8_t *msgs,
                         const uint64_t *lens, uint32_t count, uint8_t *sigs, void *stream);
hs_status hs_keyset_destroy(hs_keyset *ks);

/* Size of the fixed device buffer that hs_sign_batch_noalloc works in. */
#define HS_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)

/*
 * hs_sign_batch_noalloc -- hs_sign_batch for callers that cannot allocate
 * device memory.  The paper has no counterpart; this entry point exists for
 * users of the library.
 *
 * Who needs it: signing services that reserve all their device memory at
 * start-up and must not allocate afterwards (an allocation at peak load can
 * fail or fragment the heap), and host applications that embed this library
 * and do not let it make device allocations of its own.  hs_sign_batch takes
 * its scratch from a memory pool it creates, so those callers cannot use it.
 *
 * This variant allocates nothing: no cudaMalloc, cudaFree, pool or library
 * allocation on any call.  Its scratch is one file-scope device array of
 * HS_NOALLOC_SCRATCH_BYTES (8 MiB) that every GPU which loads this library
 * holds until the process exits.  Arguments and outputs are those of
 * hs_sign_batch, with these differences:
 *  - every buffer (sk, key_idx, msgs, lens, sigs) must be device memory of
 *    the current device: host pointers (staging them would allocate) and
 *    buffers of another GPU are rejected with HS_EINVAL; msgs may not be
 *    NULL;
 *  - a batch whose scratch does not fit the array is rejected with HS_EINVAL
 *    and hs_last_error() states the bytes needed and available.  The need is
 *    about 512 + 256 * num_keys bytes plus, per message, 1.0 KB (128f),
 *    1.4 KB (192f) or 1.8 KB (256f), so about 8000 / 5800 / 4600 messages
 *    fit.  The small-signature sets keep every leaf of their 512- or
 *    256-leaf trees in scratch: 57 KB (128s), 85 KB (192s) or 65 KB (256s)
 *    per message, so only about 140 / 95 / 125 messages fit.  The SHAKE sets
 *    need what their SHA2 counterparts need;
 *  - TREE_Sign runs chain-parallel (as hs_sign_batch does for small batches)
 *    only when its chain ends also fit the array -- 96 KB (128f), 210 KB
 *    (192f), 570 KB (256f) more per message, so up to about 80 / 38 / 14
 *    messages -- and one thread per leaf otherwise; the bytes are the same;
 *  - WOTS+_Sign recomputes its chains (no chain checkpoints are kept);
 *  - a key_idx entry >= num_keys gives an all-zero signature for that
 *    message.  It is reported through hs_check_status once the library has
 *    set up the current device (hs_keygen, hs_sign_batch or hs_check_status
 *    has run on it); before that, it is not reported.
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and caches it; make that
 * first call before any stream capture on the device.  The cached address
 * belongs to the device's current context: after cudaDeviceReset this entry
 * point (like the rest of the library) must not be used again in the
 * process.
 * All calls on a device share the one array, and it keeps the previous
 * call's contents (the call clears the words that must start at zero).
 * Calls whose work overlaps on the GPU race on the array: issue them on one
 * stream, or wait for one to finish before starting the next.
 * Signatures are byte-identical to hs_sign_batch's.
 */
hs_status hs_sign_batch_noalloc(hs_params p, const uint8_t *sk, uint32_t num_keys,
                                const uint32_t *key_idx, const uint8_t *msgs,
                                const uint64_t *lens, uint32_t count, uint8_t *sigs,
                                void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HS_H_ */
