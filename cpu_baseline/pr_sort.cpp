// Multicore CPU baseline: the paper's parallel radix-r radix sort (Section 3,
// "Parallel radix-r radix-sort", eqs. Tp, Tp4) and its two block networks for
// small n (Section 2: BTN, the bitonic merge-split network, and OET, odd-even
// transposition with merge-split; eqs. Tb and To), on std::thread workers.
//
// This is the comparison point the GPU path is measured against on the host
// cores, written independently of the serial checker and of the CUDA library.
//
// PR: p workers, worker t owns the t-th contiguous block of the input. Each
// round: every worker counts the digits of its block; the counts are
// exchanged (the paper's 2rpg term); worker t's first output position for
// digit d is (keys with a smaller digit) + (keys with digit d in blocks before
// t); every worker then routes its block's keys in input order (stable).
// BTN / OET: p blocks of ceil(n/p) items (key, original index), each sorted
// by its worker, then merge-split steps between partner blocks: the lower
// block keeps the smaller half. Items compare as (key, index), so the result
// is the stable order; padding items (key = max, index >= n) sort last.
#include <algorithm>
#include <barrier>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

template <typename K>
void pr_sort(K* keys, uint32_t* vals, size_t n, int key_bits, int rb, int p) {
    if (n < 2) return;
    if (p < 1) p = 1;
    if ((size_t)p > n) p = (int)n;
    const int bins = 1 << rb;
    std::vector<K> kb(n);
    std::vector<uint32_t> vb(vals ? n : 0);
    std::vector<size_t> cnt((size_t)p * bins);
    std::barrier sync(p);
    auto worker = [&](int t) {
        const size_t lo = n * t / p, hi = n * (t + 1) / p;
        K* src_k = keys;
        K* dst_k = kb.data();
        uint32_t* src_v = vals;
        uint32_t* dst_v = vals ? vb.data() : nullptr;
        for (int shift = 0; shift < key_bits; shift += rb) {
            const int w = std::min(rb, key_bits - shift);
            const K mask = (K)((1ull << w) - 1);
            size_t* my = cnt.data() + (size_t)t * bins;
            std::fill(my, my + bins, 0);
            for (size_t i = lo; i < hi; ++i) ++my[(src_k[i] >> shift) & mask];
            sync.arrive_and_wait();  // the count exchange
            std::vector<size_t> pos(bins);
            size_t run = 0;
            for (int d = 0; d < (1 << w); ++d) {
                for (int u = 0; u < p; ++u) {
                    if (u == t) pos[d] = run;
                    run += cnt[(size_t)u * bins + d];
                }
            }
            for (size_t i = lo; i < hi; ++i) {
                const size_t j = pos[(src_k[i] >> shift) & mask]++;
                dst_k[j] = src_k[i];
                if (vals) dst_v[j] = src_v[i];
            }
            sync.arrive_and_wait();  // the round is complete everywhere
            std::swap(src_k, dst_k);
            std::swap(src_v, dst_v);
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < p; ++t) th.emplace_back(worker, t);
    worker(0);
    for (auto& x : th) x.join();
    const int rounds = (key_bits + rb - 1) / rb;
    if (rounds % 2 == 1) {  // the result is in the scratch buffers
        std::memcpy(keys, kb.data(), n * sizeof(K));
        if (vals) std::memcpy(vals, vb.data(), n * 4);
    }
}

struct Item {
    uint32_t key, idx;
    bool operator<(const Item& o) const { return key != o.key ? key < o.key : idx < o.idx; }
};

// Merge-split of two sorted blocks of b items: x keeps the b smallest items
// of both, y the b largest (merging from the front and from the back).
void merge_split(Item* x, Item* y, size_t b, Item* tmp) {
    size_t a = 0, c = 0;
    for (size_t k = 0; k < b; ++k) tmp[k] = (c >= b || (a < b && x[a] < y[c])) ? x[a++] : y[c++];
    long long a2 = (long long)b - 1, c2 = (long long)b - 1;
    for (long long k = (long long)b - 1; k >= 0; --k)
        tmp[b + k] = (c2 < 0 || (a2 >= 0 && y[c2] < x[a2])) ? x[a2--] : y[c2--];
    std::memcpy(x, tmp, b * sizeof(Item));
    std::memcpy(y, tmp + b, b * sizeof(Item));
}

// kind 0: BTN (p a power of two, lg p (lg p + 1) / 2 steps); 1: OET (p steps).
int block_network(uint32_t* keys, uint32_t* vals, size_t n, int p, int kind) {
    if (p < 1 || (kind == 0 && (p & (p - 1)))) return 1;
    if (n < 2) return 0;
    const size_t b = (n + p - 1) / p;
    std::vector<Item> it((size_t)p * b);
    for (size_t i = 0; i < it.size(); ++i) it[i] = i < n ? Item{keys[i], (uint32_t)i} : Item{0xFFFFFFFFu, (uint32_t)i};
    // the steps: (block keeping the smaller half, block keeping the larger half)
    std::vector<std::vector<std::pair<int, int>>> steps;
    if (kind == 0) {
        for (int k = 2; k <= p; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                std::vector<std::pair<int, int>> st;
                for (int i = 0; i < p; ++i) {
                    const int q = i ^ j;
                    if (q > i) st.push_back((i & k) == 0 ? std::make_pair(i, q) : std::make_pair(q, i));
                }
                steps.push_back(st);
            }
    } else {
        for (int r = 0; r < p; ++r) {
            std::vector<std::pair<int, int>> st;
            for (int i = r & 1; i + 1 < p; i += 2) st.push_back({i, i + 1});
            steps.push_back(st);
        }
    }
    std::barrier sync(p);
    auto worker = [&](int t) {
        std::sort(it.begin() + (size_t)t * b, it.begin() + (size_t)(t + 1) * b);
        std::vector<Item> tmp(2 * b);
        sync.arrive_and_wait();
        for (const auto& st : steps) {
            for (size_t e = (size_t)t; e < st.size(); e += (size_t)p)
                merge_split(it.data() + (size_t)st[e].first * b, it.data() + (size_t)st[e].second * b, b, tmp.data());
            sync.arrive_and_wait();
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < p; ++t) th.emplace_back(worker, t);
    worker(0);
    for (auto& x : th) x.join();
    std::vector<uint32_t> v_in(vals ? vals : nullptr, vals ? vals + n : nullptr);
    for (size_t i = 0; i < n; ++i) {
        keys[i] = it[i].key;
        if (vals) vals[i] = v_in[it[i].idx];
    }
    return 0;
}

}  // namespace

extern "C" {

int cpu_pr_sort_u32(uint32_t* keys, uint32_t* vals, size_t n, int key_bits, int radix_bits, int threads) {
    if (key_bits == 0) key_bits = 32;
    if (key_bits < 1 || key_bits > 32 || radix_bits < 1 || radix_bits > 16) return 1;
    pr_sort<uint32_t>(keys, vals, n, key_bits, radix_bits, threads);
    return 0;
}

int cpu_pr_sort_u64(uint64_t* keys, uint32_t* vals, size_t n, int key_bits, int radix_bits, int threads) {
    if (key_bits == 0) key_bits = 64;
    if (key_bits < 1 || key_bits > 64 || radix_bits < 1 || radix_bits > 16) return 1;
    pr_sort<uint64_t>(keys, vals, n, key_bits, radix_bits, threads);
    return 0;
}

int cpu_btn_u32(uint32_t* keys, uint32_t* vals, size_t n, int p) { return block_network(keys, vals, n, p, 0); }
int cpu_oet_u32(uint32_t* keys, uint32_t* vals, size_t n, int p) { return block_network(keys, vals, n, p, 1); }

int cpu_hardware_threads(void) {
    const unsigned h = std::thread::hardware_concurrency();
    return h ? (int)h : 1;
}

}  // extern "C"
