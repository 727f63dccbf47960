// Tunables of the radix path (launch shapes and algorithm choices), shared by
// the single-pass rounds (radix.cu) and the chunked rounds (rts.cu).
#pragma once

#include <string>

namespace isort {

// Defaults are the measured best on GB300; the environment variable
// ISORT_TUNE ("key=value,...") overrides them.
struct Tune {
    int hist_agg = 0;     // 1: match-any aggregation in the digit histogram
    int rank_mode = 1;    // single-pass ranking: 1, per-bit ballots (the only one built)
    int shape_small = 4;  // launch shape for digits of <= 8 bits
    int shape_large = 1;  // launch shape for wider digits
    int algo = 1;         // 0: single-pass rounds with look-back, 1: chunked reduce-then-scan rounds
    int sweep_small = 4;  // chunked-round launch shape, digits of <= 8 bits, keys with payloads (4: half-warp ranking)
    int sweep_keys = 3;   // chunked-round launch shape, digits of <= 8 bits, keys only (3: per-warp masks)
    int sweep_large = 2;  // chunked-round launch shape, wider digits
    int heavy = 1;        // 1: at shape 4, a round whose digit counts have a digit over four times the mean runs
                          // the shape-3 round instead (repeated keys; picked on the device per round)
    int small = 1;        // u32 sorts of <= 65,536 keys in place at radix 2^8: one on-chip cluster launch
    int split = 8;        // chunked rounds: a digit wider than this runs as two stable passes (8..16)
    int fine = 1;         // segments of <= 8,192 keys: 1 the fine finish (two 8-bit passes + runs), 0 the older kernels
    int copy_pieces = 4;  // host-buffer staging copies: at most this many pieces on auxiliary streams
};

const Tune& tune();

// The autotuning switch of isort_autotune: true when on; *path is the cache
// file ("" for memory only).
bool autotune_config(std::string* path);
// Forgets the segmented router's tuned thresholds (isort_autotune calls it).
void router_autotune_reset();

}  // namespace isort
