/*
 * isort — GB300 (sm_103a) integer sorting: the count-sort rounds of LSD radix
 * sort, the BTN and OET block networks, a batched segmented sort and a
 * learned-bucket sort, behind a plain C ABI.
 *
 * Method: A. V. Gerbessiotis, "Integer sorting on multicores: some
 * (experiments and) observations", arXiv:1708.09495. Each entry point names the
 * section and equation that defines what it computes.
 *
 * Common conventions
 *   - Every sort is STABLE: equal keys keep their input order, so the result
 *     is the unique order by (key, original index). Keys compare as unsigned.
 *   - keys / vals are caller-owned buffers of n elements. They may live in
 *     device memory (cudaMalloc, torch tensors, managed memory) or in host
 *     memory (pinned or pageable): host buffers are staged through device
 *     memory inside the call. In the synchronous mode the call returns after
 *     the result is back in the host buffers; with isort_set_sync(0) it
 *     returns once the copies and the sort are enqueued, and the host buffers
 *     stay in use until `stream` reaches the end of that work (with pinned
 *     buffers, calls on different streams then overlap their copies in, sorts
 *     and copies out). vals == NULL means "keys only"; otherwise
 *     vals is a uint32 payload that moves with its key.
 *   - stream is a cudaStream_t (NULL = the legacy default stream). Work is
 *     enqueued on it. In the default synchronous-status mode (see
 *     isort_set_sync) the call waits for its own work to finish so that device
 *     detected errors (ISORT_ERR_KEY_RANGE, ISORT_ERR_TIMEOUT) are returned;
 *     with isort_set_sync(0) the call returns after enqueueing and those errors
 *     are collected later with isort_device_status.
 *   - Scratch memory (ping-pong buffers, digit tables, look-back words) is
 *     taken stream-ordered from a pool owned by the library on the current
 *     device and given back at the end of the call; the pool keeps the memory
 *     for reuse. ISORT_ERR_NO_MEMORY leaves the inputs untouched.
 *   - key_bits: keys must be < 2^key_bits (1..32 for u32, 1..64 for u64; 0 =
 *     full width). Fewer key bits mean fewer count-sort rounds. A key outside
 *     the range is detected before any data moves: ISORT_ERR_KEY_RANGE, buffers
 *     unchanged.
 *   - radix_bits: digit width r = 2^radix_bits, 1..16. The number of rounds is
 *     ceil(key_bits / radix_bits); the last digit is narrower when radix_bits
 *     does not divide key_bits.
 *   - n must be < 2^30 (ISORT_ERR_UNSUPPORTED otherwise). n = 0 or 1 returns
 *     ISORT_OK without touching memory.
 *   - Argument errors are reported before anything is launched.
 *   - All functions are thread-safe with respect to each other; concurrent
 *     calls on different streams use separate scratch memory.
 */
#ifndef ISORT_H_
#define ISORT_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ISORT_API __attribute__((visibility("default")))
#else
#define ISORT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ISORT_OK = 0,
    ISORT_ERR_INVALID_ARG = 1, /* a bad size, width, pointer or mode */
    ISORT_ERR_KEY_RANGE = 2,   /* some key >= 2^key_bits; buffers unchanged */
    ISORT_ERR_NO_MEMORY = 3,   /* scratch allocation failed; buffers unchanged */
    ISORT_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    ISORT_ERR_TIMEOUT = 5,     /* a bounded device wait gave up; contents unspecified */
    ISORT_ERR_UNSUPPORTED = 6  /* valid but not supported (e.g. size beyond a limit) */
} isort_status;

/* Human-readable name of a status code (static string). */
ISORT_API const char* isort_status_string(isort_status s);

/* ---------------------------------------------------------------------------
 * LSD radix sort (Section 3, "Serial/Parallel radix-r radix-sort", eqs. Ts, Tp:
 * ceil(key_bits / lg r) rounds of count-sort, least significant digit first).
 * Each round counts the digits of contiguous chunks of the keys (one read),
 * turns the counts into every chunk's output offsets (the paper's exchange of
 * counts between processors), and ranks and scatters the keys (and payloads)
 * chunk by chunk (one read, one write). Digits wider than the chunked round's
 * tables take single-pass rounds (all rounds' counts from one read, tile
 * offsets by a bounded decoupled look-back). A round of radix 2^9..2^16 (the
 * paper's r = 2^11 and 2^16 among them) runs as two stable passes over the
 * low and high halves of its digit (11 = 6 + 5, 16 = 8 + 8), which together
 * are that round's stable count-sort: a one-pass 2^16-way round would need
 * 2^16 counters per chunk, more than an SM's shared memory, and a one-pass
 * 2^11-way round measured slower than its two passes.
 * Up to 65,536 u32 keys at radix 2^8 sort in one launch: one thread-block
 * cluster (1, 2, 4 or 8 CTAs of 8,192 keys) runs every round on chip.
 * In place: on ISORT_OK keys (and vals) hold the sorted result.
 * ------------------------------------------------------------------------- */
ISORT_API isort_status isort_radix(uint32_t* keys, uint32_t* vals, size_t n, int key_bits, int radix_bits, void* stream);
ISORT_API isort_status isort_radix_u64(uint64_t* keys, uint32_t* vals, size_t n, int key_bits, int radix_bits,
                                       void* stream);

/* Out-of-place form: the inputs are read, never written; the sorted result goes
 * to keys_out / vals_out (which must not overlap the inputs). vals_in and
 * vals_out are both NULL or both non-NULL. Same rounds as isort_radix. */
ISORT_API isort_status isort_radix_copy(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                              uint32_t* vals_out, size_t n, int key_bits, int radix_bits, void* stream);
ISORT_API isort_status isort_radix_copy_u64(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                  uint32_t* vals_out, size_t n, int key_bits, int radix_bits, void* stream);

/* ---------------------------------------------------------------------------
 * Typed keys. The paper sorts unsigned integers; signed integers and IEEE 754
 * floats are sorted by the same rounds through an order-preserving map of
 * their bits, applied in place before the rounds and undone after them:
 * signed: flip the sign bit; float: flip every bit of a key whose sign bit is
 * set, else only the sign bit. Orders: integers by value; floats by IEEE 754
 * totalOrder (-NaN < -Inf < ... < -0 < +0 < ... < +Inf < +NaN; NaNs by their
 * payload bits). Stable: equal keys (same bits) keep their input order.
 * key_type: ISORT_KEY_U32, _I32, _F32 (4-byte keys), _U64, _I64, _F64
 * (8-byte keys); keys and vals (optional u32 payload) are DEVICE memory,
 * sorted in place over the full key width; radix_bits 1..16.
 * ------------------------------------------------------------------------- */
enum { ISORT_KEY_U32 = 0, ISORT_KEY_I32 = 1, ISORT_KEY_F32 = 2, ISORT_KEY_U64 = 3, ISORT_KEY_I64 = 4, ISORT_KEY_F64 = 5 };
ISORT_API isort_status isort_radix_typed(void* keys, int key_type, uint32_t* vals, size_t n, int radix_bits,
                                         void* stream);

/* ---------------------------------------------------------------------------
 * The two primitives of a count-sort round (Section 3, "Serial radix-r"), for
 * callers that drive rounds themselves and for checking each step.
 *
 * isort_digit_hist: hist[d * 2^radix_bits + b] = number of keys whose round-d
 *   digit (key >> d*radix_bits) & (2^w - 1) equals b, for every round d <
 *   ceil(key_bits / radix_bits) (w = radix_bits, or what is left of key_bits in
 *   the last round). hist is a DEVICE buffer of rounds * 2^radix_bits uint32
 *   that the call overwrites. keys is device memory. key_width is 32 or 64.
 *   Key range violations are reported as ISORT_ERR_KEY_RANGE (hist still
 *   written).
 * isort_count_round: one stable count-sort round on the digit
 *   (key >> shift) & (2^width - 1), width 1..16, out of place: the output is
 *   ordered by digit, ties in input order. All buffers are device memory.
 * ------------------------------------------------------------------------- */
ISORT_API isort_status isort_digit_hist(const void* keys, int key_width, size_t n, int key_bits, int radix_bits,
                              uint32_t* hist, void* stream);
ISORT_API isort_status isort_count_round(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                               uint32_t* vals_out, size_t n, int shift, int width, void* stream);
ISORT_API isort_status isort_count_round_u64(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                   uint32_t* vals_out, size_t n, int shift, int width, void* stream);

/* ---------------------------------------------------------------------------
 * BTN (Section 2 and Section 3 "Bitonic Sort", eq. Tb): the n keys are split
 * into p blocks of ceil(n/p), each block is sorted locally, then a p-input
 * bitonic network of lg p (lg p + 1)/2 stages runs with every comparator
 * replaced by a merge-split (the lower block keeps the smaller half).
 * OET (Section 2 and Section 3 "Odd-even transposition sort", eq. To): the same
 * p sorted blocks, then p rounds of merge-split between neighbouring blocks
 * (j, j+1), j = round mod 2.
 * Items compare as (key, original index), which makes the networks stable.
 * On the GPU a block lives in one thread's registers; one CTA sorts the array.
 * isort_btn / isort_oet choose p; the _p forms take it (BTN: a power of two
 * 1..1024; OET: 1..1024) and, if stages != NULL, store the number of
 * merge-split stages / rounds executed in *stages (host memory).
 * Limits: one CTA holds the p blocks: n <= 16384, at most 32 keys per block
 * (n <= 32 * p), and at most 16 keys per block when p > 512. Other sizes give
 * ISORT_ERR_UNSUPPORTED.
 * ------------------------------------------------------------------------- */
ISORT_API isort_status isort_btn(uint32_t* keys, uint32_t* vals, size_t n, void* stream);
ISORT_API isort_status isort_oet(uint32_t* keys, uint32_t* vals, size_t n, void* stream);
ISORT_API isort_status isort_btn_p(uint32_t* keys, uint32_t* vals, size_t n, int p, uint64_t* stages, void* stream);
ISORT_API isort_status isort_oet_p(uint32_t* keys, uint32_t* vals, size_t n, int p, uint64_t* stages, void* stream);

/* ---------------------------------------------------------------------------
 * Batched segmented sort: segment s is keys[seg_offsets[s] .. seg_offsets[s+1])
 * (with the same range of vals); every segment is sorted stably and in place,
 * independently of the others. One launch sequence, captured in a CUDA graph,
 * serves all segments; each segment is routed on the device by its length to
 * OET (Section 2; <= 32 keys, one warp), BTN (Section 2, eq. Tb; <= 256 keys in
 * one warp, <= 4096 keys in one CTA) or count-sort rounds of 8-bit digits
 * (Section 3, eq. Ts) run entirely on chip: up to 8,192 keys by one CTA (two
 * passes over the top 16 bits of the segment's observed key range, then runs
 * of equal top bits sorted on the low bits), up to 65,536 keys by a cluster of
 * 2, 4 or 8 CTAs. The cut-offs given are the built-in ones; with
 * isort_autotune on, the network cut-offs are measured on the GPU once and
 * cached. Longer segments use isort_radix's rounds, one segment at a
 * time; in the asynchronous status mode or while `stream` is being captured
 * they are not supported (ISORT_ERR_UNSUPPORTED recorded).
 * keys, vals (may be NULL) and seg_offsets (nseg + 1 uint64, non-decreasing)
 * are device memory. key_bits as for isort_radix; a segment holding a key
 * >= 2^key_bits is left unchanged and ISORT_ERR_KEY_RANGE is returned; other
 * segments are still sorted. Decreasing offsets: ISORT_ERR_INVALID_ARG (those
 * segments are skipped). nseg < 2^31.
 * ------------------------------------------------------------------------- */
ISORT_API isort_status isort_segmented(uint32_t* keys, uint32_t* vals, const uint64_t* seg_offsets, size_t nseg,
                                       int key_bits, void* stream);

/* ---------------------------------------------------------------------------
 * Learned-bucket sort. The paper has no counterpart; it grows out of the
 * splitter-based sample sorts the paper discusses (Section 2: oversampling and
 * regular sampling), with the splitters read off a learned CDF, and finishes
 * buckets with the count-sort rounds of Section 3. One call:
 *   1. samples 2^16 keys (indices from SplitMix64 seeded with 0x5EED5EED5EED:
 *      index_j = floor(r_j * n / 2^64)) and sorts them with the radix rounds;
 *   2. trains a monotone piecewise-linear CDF F over u = key * 2^-key_bits
 *      (256 segments; knots X_0..X_256 and values Y_0..Y_256 are normalised
 *      cumulative sums of softplus(theta), so F is monotone by construction;
 *      knots start at the sample's quantiles) by 64 Adam steps on
 *      (1/m) sum_i (F(u_i) - (i + 1/2)/m)^2 over every 8th point of the
 *      sorted sample (m = 2^13), on the GPU;
 *   3. gives every key the bucket min(B - 1, floor(F(u) B)), F evaluated in a
 *      fixed fp32 order and clamped to each segment's value range, which makes
 *      the bucket monotone in the key (buckets are key ranges); the splitter
 *      table s_b = the first key of bucket b gives each bucket's key range;
 *   4. distributes the keys stably by bucket (the bucket of every key is
 *      computed once and stored as 16 bits, which move with the key through
 *      the two passes over the id's halves) and sorts every bucket on chip on
 *      the bits its key range spans (a bucket of one key value is skipped).
 * The output is the stable sort of the input, whatever the model learned.
 * keys (u32), vals (optional) are device memory; nbuckets 2..32768 (0 = 4096,
 * doubled up to 32768 while n / nbuckets > 16,384; for u64 keys the smallest
 * multiple of 4096 whose mean bucket holds at most 6,656 keys, up to 32768);
 * model 0 = the piecewise-linear CDF of step 2; model 1 = a 1-32-1 monotone
 * MLP CDF instead (see isort_mlp_train), trained on every 16th point of the
 * sorted sample and tabulated as the 257 knots (X_k, Y_k) steps 3-4 read;
 * model 2 = no training (the method without a learned model): the table of
 * step 2's start, knots at the sample's quantiles j/256 with values j/256,
 * i.e. regular sampling (Section 2) with 255 evenly spaced sample keys as
 * splitters, each interval split evenly in key space when nbuckets > 256.
 * n < 2^18 sorts with the plain rounds. If more than half of the keys fall in
 * buckets beyond the on-chip capacity (65,536 keys) the call sorts with the
 * plain rounds instead (stats->fell_back_to_lsd = 1); fewer such buckets are
 * gathered into one buffer (their key ranges are disjoint and ordered), sorted
 * by one call of the plain rounds and scattered back. The call synchronizes
 * (the bucket sizes are read on the host). stats (host, may be NULL) receives
 * the bucket balance and the training record.
 * ------------------------------------------------------------------------- */
typedef struct {
    double imbalance_max_over_mean; /* largest bucket / (n / nbuckets) */
    double overflow_fraction;       /* keys in buckets over 65,536 keys / n */
    uint64_t fixups;                /* 0: the bucket function needs no corrections (kept for layout) */
    uint64_t overflow_buckets;      /* buckets over 65,536 keys */
    int fell_back_to_lsd;           /* 1: sorted by the plain rounds */
    int train_steps;
    float train_loss_initial;       /* sample loss before training */
    float train_loss;               /* sample loss after training */
    int nbuckets;
} isort_learned_stats;
ISORT_API isort_status isort_learned(uint32_t* keys, uint32_t* vals, size_t n, int key_bits, int nbuckets, int model,
                                     isort_learned_stats* stats, void* stream);
/* The same for u64 keys (key_bits 1..64, 0 = 64; u = key * 2^-key_bits). The
 * sample is sorted as one on-chip segment; buckets of up to 8,192 keys are
 * finished by two on-chip 8-bit passes over the top 16 bits of their observed
 * key range (runs of equal top bits then sorted on the low bits), larger ones
 * by the on-chip split on packed 64-bit items. */
ISORT_API isort_status isort_learned_u64(uint64_t* keys, uint32_t* vals, size_t n, int key_bits, int nbuckets,
                                         int model, isort_learned_stats* stats, void* stream);

/* The learned path's steps, for callers that drive them and for checking:
 * isort_cdf_train: trains the model on a sorted sample (device, m u32 keys):
 *   theta (device, 512 floats: 256 knot increments then 256 value
 *   increments), X and Y (device, 257 floats each) receive the trained model
 *   (the parameters with the lowest sample loss seen, the initial ones
 *   included); losses (device, 66 floats) the loss before each of the 64
 *   steps, then the loss of the returned model, then the loss at the initial
 *   parameters.
 * isort_cdf_loss_grad: loss and d loss / d theta at theta (device, 512) on
 *   u (device, m normalised sorted sample values); grad (device, 512) and
 *   loss (device, 1) receive them.
 * isort_cdf_splitters: the splitter table of step 3 from X, Y (device, 257
 *   floats each): splitters (device, nbuckets entries of key_width bits,
 *   nbuckets 2..65536; entry 0 is 0; s_b = the first key of bucket b).
 * isort_bucket_ids: the bucket of step 3 of every key (device, key_width 32
 *   or 64) given X, Y (nbuckets 2..65536); ids (device, n uint32, n < 2^32).
 */
ISORT_API isort_status isort_cdf_train(const uint32_t* sorted_sample, uint32_t m, int key_bits, float* theta, float* X,
                                       float* Y, float* losses, void* stream);
ISORT_API isort_status isort_cdf_loss_grad(const float* u, uint32_t m, const float* theta, float* grad, float* loss,
                                           void* stream);
ISORT_API isort_status isort_cdf_splitters(const float* X, const float* Y, int key_width, int key_bits, int nbuckets,
                                           void* splitters, void* stream);
ISORT_API isort_status isort_bucket_ids(const void* keys, int key_width, size_t n, int key_bits, const float* X,
                                        const float* Y, int nbuckets, uint32_t* ids, void* stream);

/* The MLP model (isort_learned with model = 1). Parameters (device, 97
 * floats): a1[32], b1[32], a2[32], b2, with W1 = softplus(a1),
 * W2 = softplus(a2),
 *   z(u) = sum_j W2_j sigmoid(W1_j u + b1_j) + b2,
 *   F(u) = (z(u) - z(0)) / (z(1) - z(0)),
 * increasing with F(0) = 0, F(1) = 1 (b2 cancels). Same loss as step 2.
 * isort_mlp_train: from a sorted sample (device, m u32 keys) sets the initial
 *   parameters (unit j centred at the sample's (j + 1/2)/32 quantile, rising
 *   over its quantile interval; W2 = 1/32), runs 64 Adam steps on one
 *   cluster of 8 CTAs over all m points, and writes params (the lowest loss
 *   seen), X, Y (device, 257 each: X_0 = 0, X_k = the normalised key of rank
 *   k m / 256, X_256 = 1; Y_k = F(X_k) clamped to [0, 1] and made
 *   non-decreasing, Y_0 = 0, Y_256 = 1) and losses (device, 66 floats, laid
 *   out as for isort_cdf_train).
 * isort_mlp_loss_grad: loss and d loss / d params at params (device, 97) on
 *   u (device, m normalised sorted values); grad (device, 97; the b2 entry is
 *   0) and loss (device, 1) receive them.
 */
ISORT_API isort_status isort_mlp_train(const uint32_t* sorted_sample, uint32_t m, int key_bits, float* params, float* X,
                                       float* Y, float* losses, void* stream);
ISORT_API isort_status isort_mlp_loss_grad(const float* u, uint32_t m, const float* params, float* grad, float* loss,
                                           void* stream);

/* ---------------------------------------------------------------------------
 * Sample-sort steps for a sort spread over p processes (Section 2, the sample
 * sorts with regular sampling; the routing of keys is Section 3's count-sort
 * round with the key's range as its digit, the key exchange of eq. Tp).
 *
 * isort_sample: out[j] = keys[floor(r_j * n / 2^64)] for j < m, r_j the j-th
 *   output of SplitMix64 started at state `seed` (Steele, Lea & Flood 2014).
 *   key_width 32 (uint32 keys) or 64 (uint64 keys); keys (n >= 1) and out (m
 *   keys) are device memory, owned by the caller. m = 0 is a no-op.
 *   ISORT_ERR_INVALID_ARG for another key width, n = 0 with m > 0, NULL or
 *   host pointers.
 * isort_partition[_u64]: the stable routing of n keys (and payloads) into
 *   `parts` ranges. Splitter j (1 <= j < parts) is
 *   sorted_sample[floor(j * m / parts)] (a regular choice among m sample keys
 *   sorted ascending, e.g. the samples of all processes gathered and sorted);
 *   the range of a key is the number of splitters <= key. keys_out/vals_out
 *   receive range 0's keys, then range 1's, ..., each in input order;
 *   counts[r] (uint64, `parts` entries) = keys in range r. All pointers are
 *   device memory owned by the caller; the output must not overlap the input
 *   (vals: both or neither). parts in 1..256 (m >= 1 when parts > 1);
 *   n < 2^32 (larger: ISORT_ERR_UNSUPPORTED). ISORT_ERR_INVALID_ARG for other
 *   values, NULL, host or aliased pointers. Scratch as isort_radix.
 * ------------------------------------------------------------------------- */
ISORT_API isort_status isort_sample(const void* keys, int key_width, size_t n, uint32_t m, uint64_t seed, void* out,
                                    void* stream);
ISORT_API isort_status isort_partition(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                       uint32_t* vals_out, size_t n, const uint32_t* sorted_sample, size_t m,
                                       int parts, uint64_t* counts, void* stream);
ISORT_API isort_status isort_partition_u64(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                           uint32_t* vals_out, size_t n, const uint64_t* sorted_sample, size_t m,
                                           int parts, uint64_t* counts, void* stream);

/* ---------------------------------------------------------------------------
 * isort_radix_noalloc: isort_radix (in place, u32 keys, optional u32 payload)
 * for callers that must not allocate memory. The paper has no counterpart; it
 * exists because some callers cannot let a library allocate device memory:
 * processes whose device memory is reserved up front by another allocator,
 * and latency-critical loops that cannot take the implicit synchronisation of
 * an allocation.
 * It allocates nothing: all scratch comes from one 5 MiB array in device
 * memory that the library declares at file scope; every GPU that loads the
 * library holds that array until the process exits. Limits: n <= 262,144 keys
 * and radix_bits <= 8 (larger: ISORT_ERR_UNSUPPORTED); keys and vals must be
 * device memory (host pointers: ISORT_ERR_INVALID_ARG). Other arguments,
 * results and errors are those of isort_radix.
 * The first call on a device looks up the array's device address for that
 * device (cudaGetSymbolAddress, with the device current). All calls on a
 * device share the array and
 * it keeps the last call's contents: calls whose work overlaps on the GPU
 * (different streams, or several calls enqueued in the asynchronous status
 * mode before the earlier ones finished) race and corrupt each other's
 * results. In the synchronous status mode the call waits for `stream` and
 * returns device-detected errors; on a stream that reports an active capture
 * it does not wait, and device-detected errors are recorded as in the
 * asynchronous mode (read them with isort_device_status).
 * ------------------------------------------------------------------------- */
ISORT_API isort_status isort_radix_noalloc(uint32_t* keys, uint32_t* vals, size_t n, int key_bits, int radix_bits,
                                           void* stream);

/* ---------------------------------------------------------------------------
 * Status mode and device-side checks.
 * isort_set_sync(1) (default): calls wait for their work and return device
 *   detected errors. isort_set_sync(0): calls return after enqueueing.
 * isort_device_status: waits for `stream`, returns the first device-detected
 *   error recorded by asynchronous calls on the current device since the last
 *   clear (ISORT_OK if none), and clears it when clear != 0.
 * isort_set_spin_limit: upper bound, in microseconds, of every device-side
 *   wait (look-back, copy completion). A wait that runs out records
 *   ISORT_ERR_TIMEOUT and the kernel returns. Default 2,000,000 (2 s).
 * ------------------------------------------------------------------------- */
/* Autotuning (the library's own choices, not in the paper). enable = 1:
 * - the count-sort rounds' launch shape: the first radix sort of each kind
 *   (key width, payload or not, digits of <= 8 bits or wider, floor(log2 n);
 *   n >= 2^20) times the candidate shapes once on synthetic keys of the same
 *   size and keeps the fastest ("key_bytes payload wide log2n shape" lines);
 * - the segmented router's length cut-offs between OET in a warp, BTN in a
 *   warp, BTN over a CTA and the on-chip count-sort rounds (Section 4,
 *   Observations 5-6: the networks win for small n): the first segmented sort
 *   of each kind (keys only, with payloads) times every method on batches of
 *   equal-length segments of 8..4096 keys and takes as each cut-off the
 *   largest length at which that method was the fastest ("router payload oet
 *   btn_warp btn_cta" lines; the built-in cut-offs are 32, 256, 4096).
 * Timing allocates scratch and synchronises the stream; inside a stream
 * capture the built-in (or cached) choices are used. Choices last for the
 * process, are read from cache_path (text; NULL: memory only) and appended to
 * it. enable = 0: the built-in choices. ISORT_ERR_INVALID_ARG for other
 * values of enable. The sorted output never depends on these choices. */
ISORT_API isort_status isort_autotune(int enable, const char* cache_path);

ISORT_API isort_status isort_set_sync(int on);
ISORT_API isort_status isort_device_status(int clear, void* stream);
ISORT_API isort_status isort_set_spin_limit(uint64_t microseconds);

/* ---------------------------------------------------------------------------
 * Fault injection for tests: isort_debug_stall_tile(t) makes the next radix
 * sort run its rounds in the single-pass form (tiles resolve their offsets by
 * looking back at earlier tiles' published counts) with tile t of the first
 * round never publishing, so that its successors' waits run out (t < 0
 * disables). It only ever causes bounded waits.
 * ------------------------------------------------------------------------- */
ISORT_API isort_status isort_debug_stall_tile(int64_t tile);

/* ---------------------------------------------------------------------------
 * Introspection.
 * isort_launch_count: number of kernels this library has launched so far in
 *   this process. isort_last_error_string: see its declaration.
 * isort_profile_enable(1): record CUDA events around every kernel launch.
 * isort_profile_read: waits for the recorded events, writes up to max entries
 *   (one per kernel name: launches and total milliseconds) and clears the
 *   record; returns the number of entries written.
 * ------------------------------------------------------------------------- */
ISORT_API uint64_t isort_launch_count(void);
/* Text of the last CUDA error or device-side status this thread's calls met
 * ("" if none); valid until the thread's next call. */
ISORT_API const char* isort_last_error_string(void);
typedef struct {
    char name[48];
    uint64_t launches;
    double total_ms;
} isort_kernel_time;
ISORT_API isort_status isort_profile_enable(int on);
ISORT_API int isort_profile_read(isort_kernel_time* out, int max);

#ifdef __cplusplus
}
#endif
#endif /* ISORT_H_ */
