// hs_launch.h -- host-side launchers of the signer's kernels (library
// internal; the public surface is include/hs.h).  Each launcher dispatches
// on the parameter set id (0 128f, 1 192f, 2 256f, 3 toy, 4-6 128s-256s,
// 7-12 the SHAKE instantiations of 0-2 and 4-6) to the kernel template
// instantiated for that set.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include "hs_params.cuh"

namespace hs {

// A distinct XMSS tree of a batch (tree sharing, kern_dedup.cuh).
struct DedupDesc {
    uint64_t tree;
    uint32_t key;
    uint32_t layer;
};

// Device buffers of one sign or verify call.  'sk' is the caller's key
// buffer for signing (4n bytes per key) or public keys for verifying (2n).
struct Batch {
    int pset;
    const uint8_t* keys_in;   // sk (sign) or pk (verify), num_keys entries
    uint32_t num_keys;
    const uint32_t* key_idx;  // may be null: key 0
    const uint8_t* msgs;
    const uint64_t* lens;
    uint32_t count;
    uint8_t* sigs;            // sign: out; verify: in (const)
    uint8_t* ok;              // verify only
    bool verify;              // a verification call (scratch: chain ends of one layer)
    uint32_t* vcnt;           // verify: 16 chain-length buckets per layer (16 D words)
    uint32_t* vsitem;         // verify: count * LEN words, steps << 28 | rank
    uint32_t* vorder;         // verify: count * LEN words, chains sorted by length
    // scratch
    KeyBlock* keys;           // num_keys
    uint64_t* offsets;        // count + 1
    MsgInfo* infos;           // count
    uint32_t* fors_roots;     // count * K * NW words
    uint32_t* pk_fors;        // count * NW words
    uint32_t* roots;          // count * D * NW words
    uint32_t* chk;            // WOTS chain checkpoints: count * D * LEN * (16 / ck) * NW words
    uint32_t ck;              // checkpoint stride (1, 2, 4) or 0 = none
    bool split;               // TREE_Sign in its chain-parallel form (small batches)
    uint32_t* ends;           // chain ends of the split form: count * D * 2^h' * LEN * NW words
    uint32_t* leafv;          // wide trees (2^h' > 32): leaves, count * D * 2^h' * NW words
    // tree sharing within the batch: layers dedup_layer .. D-1 are shared
    // (dedup_layer == 0: off, every message builds all its layers)
    uint32_t dedup_layer;
    uint32_t cap_log2;        // hash table of 2^cap_log2 slots
    uint32_t max_uniq;        // bound on the distinct trees
    unsigned long long* table;
    uint32_t* mj_slot;        // count * (D - L)
    uint32_t* mj_id;          // count * (D - L)
    uint32_t* slot_id;        // 2^cap_log2
    uint32_t* nuniq;
    DedupDesc* desc;          // max_uniq
    uint32_t* nodes_u;        // max_uniq * 2 * 2^h' * NW words
    uint32_t* chk_u;          // max_uniq * 2^h' * LEN * (16 / ck) * NW words
    // keyset cache: layers dedup_layer .. D-1 come prebuilt from nodes_u /
    // chk_u (owned by the keyset), tree ids computed directly (no table)
    bool cached;
    uint32_t cache_tpk;       // cached trees per key
    // FIPS 205 mode: FORS indices MSB first; prefix bytes hashed before
    // every message (0x00 || len(ctx) || ctx for pure signing; none = 0)
    bool fips;
    const uint8_t* prefix;    // device, prefix_len bytes
    uint32_t prefix_len;
    uint32_t* status;         // per-device status word
    // message stage: a warp per message (SHA-2 sets, small batches; the
    // form is fixed with the batch, like 'split')
    bool msg_warp;
};

// Record the text hs_last_error() returns on the calling thread.
void set_last_error(const char* msg);

// Library state shared by the entry points: the current device's status
// word (nullptr if the device state could not be set up), a stream-ordered
// allocation from the library's pool, and the chain checkpoint stride.
uint32_t* device_status_word();
// The same word if the library has already set up the current device, else
// nullptr; never allocates.
uint32_t* device_status_word_if_ready();
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s);
uint32_t chain_checkpoint_stride(int pset);

// Tree sharing plan of a batch: fills dedup_layer, cap_log2 and max_uniq
// (dedup_layer = 0 when sharing is off or not worth it).
void plan_dedup(Batch& b);
size_t scratch_bytes(const Batch& b);

// Scratch bytes for a batch (each region 256-byte aligned).
// cached_from: first layer taken from a keyset's cache (0 = none).
size_t scratch_bytes(int pset, uint32_t num_keys, uint32_t count, uint32_t ck, bool split = false,
                     uint32_t cached_from = 0);
void carve_scratch(Batch& b, void* base);

// Per-parameter-set kernel launchers (one table per set_<name>.cu).  The
// FORS and TREE launchers take the tuned launch shape: lanes per FORS tree
// and the minimum resident blocks per SM of TREE_Sign (0 = compiler choice);
// the arrays list the compiled variants, the *_default fields the defaults.
struct SetOps {
    cudaError_t (*keyprep)(const Batch&, bool, cudaStream_t);
    cudaError_t (*message)(const Batch&, bool, cudaStream_t);
    cudaError_t (*fors)(const Batch&, int, cudaStream_t);
    cudaError_t (*fors_pk)(const Batch&, cudaStream_t);
    // TREE_Sign per leaf: (min blocks, addition policy, chains per thread);
    // tree_has says which combinations are compiled
    cudaError_t (*tree)(const Batch&, int, int, int, cudaStream_t);
    bool (*tree_has)(int, int, int);
    cudaError_t (*tree_split)(const Batch&, cudaStream_t);
    cudaError_t (*tree_dedup)(const Batch&, cudaStream_t);
    cudaError_t (*tree_cached)(const Batch&, cudaStream_t);
    cudaError_t (*cache_build)(const KeyBlock*, uint32_t, uint32_t, uint32_t, DedupDesc*, uint32_t*, uint32_t*,
                               uint32_t, cudaStream_t);
    cudaError_t (*wots)(const Batch&, cudaStream_t);
    cudaError_t (*verify)(const Batch&, cudaStream_t);
    cudaError_t (*keygen)(const uint8_t*, uint32_t, uint8_t*, uint8_t*, cudaStream_t);
    const int* fors_lpt;
    int n_fors_lpt;
    int fors_lpt_default;
    const int* tree_minb;
    int n_tree_minb;
    int tree_minb_default;
    int tree_pol_default;
};
extern const SetOps kOps_128F, kOps_192F, kOps_256F, kOps_Toy, kOps_128S, kOps_192S, kOps_256S;
extern const SetOps kOps_K128F, kOps_K192F, kOps_K256F, kOps_K128S, kOps_K192S, kOps_K256S;
extern const SetOps kOps_R128F, kOps_R192F, kOps_R256F;
// 128f, 192f, 256f, toy, 128s, 192s, 256s, then the SHAKE instantiations of
// 128f .. 256s, then the robust SHA2 instantiations of 128f, 192f, 256f
constexpr int kNumSets = 16;

// Shape of a parameter set for host code (false for an unknown id).
struct SetShape { int n, d, sig, leaves, k; };
bool set_shape(int pset, SetShape* out);
const SetOps* set_ops(int pset);

// Tuned launch shape per set (knob 0 = FORS lanes per tree, 1 = TREE min
// blocks, 2 = batch size below which TREE_Sign runs chain-parallel, 3 =
// TREE_Sign addition policy, 4 = TREE_Sign chains per thread, 5 = chain
// checkpoint stride, 6 = per-leaf TREE_Sign time of one warp per SM
// sub-partition (us), 7 = chain-parallel TREE_Sign time per message (ns),
// 8 = batch size below which the message stage runs a warp per message).
constexpr int kNumKnobs = 9;
int tune_get(int pset, int knob);
bool tune_set(int pset, int knob, int value);
// Compiled values of a knob (returns how many; -1 for bad arguments).
int tune_options(int pset, int knob, int32_t* values, int max);
// Process-wide checkpoint stride: the value of every set whose knob 5 is unset.
void set_default_checkpoint(uint32_t stride);
bool tree_split(int pset, uint32_t count);
// Whether a batch's message stage runs a warp per message (knob 8).
bool msg_warp(int pset, uint32_t count);
// SM count of the current device (cached per device).
int sm_count();
// Lanes per FORS tree for a batch of 'count' messages: the tuned value, or
// for a batch too small to give the launch about 1024 threads per SM, the
// next wider compiled lane groups (fewer leaves per lane, same bytes).
int fors_lanes(int pset, uint32_t count);

cudaError_t launch_keyprep(const Batch& b, bool from_pk, cudaStream_t s);
cudaError_t launch_offsets(const Batch& b, cudaStream_t s);
cudaError_t launch_message(const Batch& b, bool verify, cudaStream_t s);
cudaError_t launch_fors(const Batch& b, cudaStream_t s);
cudaError_t launch_fors_pk(const Batch& b, cudaStream_t s);
cudaError_t launch_tree(const Batch& b, cudaStream_t s);
cudaError_t launch_wots(const Batch& b, cudaStream_t s);
cudaError_t launch_verify(const Batch& b, cudaStream_t s);
cudaError_t launch_keygen(int pset, const uint8_t* seeds, uint32_t count, uint8_t* pk, uint8_t* sk,
                          cudaStream_t s);

}  // namespace hs

// A keyset (include/hs.h): resident keys and the prebuilt trees of their top
// layers, shared by hs_sign_keyset and the server.
struct hs_keyset {
    int pset = 0;
    int device = 0;
    uint32_t num_keys = 0;
    uint32_t layers = 0;        // cached top layers
    uint32_t first_layer = 0;   // d - layers
    uint32_t tpk = 0;           // cached trees per key
    uint32_t ck = 0;            // chain checkpoint stride of the cache
    uint8_t* sk = nullptr;      // num_keys * 4n bytes
    hs::KeyBlock* kb = nullptr; // num_keys
    uint32_t* nodes = nullptr;  // trees * 2 * 2^h' * NW words, heap order per tree
    uint32_t* chk = nullptr;    // trees * 2^h' * len * (16 / ck) * NW words (ck != 0)
    size_t bytes = 0;
};
