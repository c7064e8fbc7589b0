// Oracle for the PI batch path: a plain, sequential pointer skip list.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call this
// file; only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
// It shares no code, header, table or constant generator with the CUDA library.
//
// What it computes (the definition the GPU path must reach exactly):
//   * PI claims serializable batches (Section 4.2, "only one thread takes charge of each
//     data node at any time"), so a batch is equal to applying its queries one at a time
//     in arrival order to a dictionary key -> value. execute() does exactly that with a
//     for-loop over the queries.
//   * Each query reports the state of its key just before it runs: PRESENT with the
//     value, or ABSENT with value 0. For a search this is Algorithm 4's result (return
//     the node's pointer if the key matches and the delete flag is clear, else null).
//     For a delete, PRESENT is the "return 1" of the Delete definition (Section 3.2).
//     For an insert the paper returns null; returning the prior state is this
//     library's extension, and it is fully determined by the same replay.
//   * Insert overwrites the value of an existing key or adds the key (Section 3.2,
//     Insert). Delete removes the key (Section 3.2, Delete).
//   * A query whose op code is not 0/1/2 or whose key is 2^64-1 (reserved) is INVALID
//     and has no effect.
//   * The structure (Section 3.1, Definition 1): level 1 holds every live key; level l
//     holds the live keys whose tower height is at least l. The height replaces the
//     paper's geometric draw with a seeded hash of the key:
//         h = splitmix64(key ^ splitmix64(seed))
//         height = 1 + min(ctz(h) / b, Hmax - 1),  p = 2^-b,  Hmax = min(32, 64 / b)
//     with ctz(0) = 64. P(height >= l) = p^(l-1), as for the geometric draw.
//
// Mechanism: a Pugh skip list (the structure PI extends, Section 2): each node has a
// key, a value and `height` forward pointers. Searches walk from the head, top level
// down. Deletes unlink and discard the node (physical removal; no delete flag), so the
// oracle does not mirror the GPU design's tombstones. Bulk construction links a sorted
// input level by level in one pass (Section 3.1: the index is built bottom-up by one
// scan of the storage layer). Nodes come from an arena that is released on destroy.

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

namespace {

constexpr uint64_t kReservedKey = ~0ull;
constexpr int kMaxLevels = 32;

// SplitMix64 (Steele, Lea and Flood 2014): one generator step from state x.
uint64_t oracle_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int count_trailing_zeros(uint64_t h) {
    if (h == 0) return 64;
    int c = 0;
    while ((h & 1ull) == 0) {
        h >>= 1;
        ++c;
    }
    return c;
}

struct Node {
    uint64_t key;
    uint64_t value;
    int height;
    Node* next[1];  // really `height` entries
};

struct Arena {
    std::vector<char*> blocks;
    size_t used = 0, cap = 0;
    void* take(size_t bytes) {
        bytes = (bytes + 15) & ~size_t(15);
        if (used + bytes > cap) {
            size_t sz = std::max<size_t>(bytes, size_t(64) << 20);
            char* b = static_cast<char*>(std::malloc(sz));
            if (!b) throw std::bad_alloc();
            blocks.push_back(b);
            used = 0;
            cap = sz;
        }
        void* p = blocks.back() + used;
        used += bytes;
        return p;
    }
    ~Arena() {
        for (char* b : blocks) std::free(b);
    }
};

struct SkipList {
    int b = 1;              // p = 2^-b
    int hmax = 32;          // min(32, 64 / b)
    uint64_t seed_mix = 0;  // splitmix64(seed)
    uint64_t count = 0;     // live keys
    Node* head = nullptr;   // sentinel with hmax forward pointers
    Arena arena;

    int height_of(uint64_t key) const {
        uint64_t h = oracle_splitmix64(key ^ seed_mix);
        int lvl = count_trailing_zeros(h) / b;
        if (lvl > hmax - 1) lvl = hmax - 1;
        return 1 + lvl;
    }

    Node* new_node(uint64_t key, uint64_t value) {
        int h = height_of(key);
        size_t bytes = sizeof(Node) + sizeof(Node*) * (h - 1);
        Node* n = static_cast<Node*>(arena.take(bytes));
        n->key = key;
        n->value = value;
        n->height = h;
        for (int i = 0; i < h; ++i) n->next[i] = nullptr;
        return n;
    }

    void init(int b_, uint64_t seed) {
        b = b_;
        hmax = std::min(32, 64 / b);
        seed_mix = oracle_splitmix64(seed);
        size_t bytes = sizeof(Node) + sizeof(Node*) * (kMaxLevels - 1);
        head = static_cast<Node*>(arena.take(bytes));
        head->key = 0;
        head->value = 0;
        head->height = kMaxLevels;
        for (int i = 0; i < kMaxLevels; ++i) head->next[i] = nullptr;
    }

    // Top-down search. update[i] = last node at level i+1 whose key is < key.
    Node* find(uint64_t key, Node** update) const {
        Node* x = head;
        for (int i = hmax - 1; i >= 0; --i) {
            while (x->next[i] && x->next[i]->key < key) x = x->next[i];
            update[i] = x;
        }
        Node* c = x->next[0];
        return (c && c->key == key) ? c : nullptr;
    }

    void insert_or_assign(uint64_t key, uint64_t value, Node** update) {
        Node* n = new_node(key, value);
        for (int i = 0; i < n->height; ++i) {
            n->next[i] = update[i]->next[i];
            update[i]->next[i] = n;
        }
        ++count;
    }

    void unlink(Node* n, Node** update) {
        for (int i = 0; i < n->height; ++i) {
            if (update[i]->next[i] == n) update[i]->next[i] = n->next[i];
        }
        --count;  // the node's memory stays in the arena until destroy
    }
};

}  // namespace

extern "C" {

enum { O_ABSENT = 0, O_PRESENT = 1, O_INVALID = 2 };

uint64_t osl_splitmix64(uint64_t x) { return oracle_splitmix64(x); }

int osl_height(uint64_t seed, int b, uint64_t key) {
    SkipList s;
    s.b = b;
    s.hmax = std::min(32, 64 / b);
    s.seed_mix = oracle_splitmix64(seed);
    return s.height_of(key);
}

// Builds from (keys, values); a key that appears more than once keeps its LAST value,
// as if the pairs were inserted in order. Returns nullptr and sets *err on bad input:
// -1 for a bad promotion exponent or the reserved key, -2 on allocation failure.
void* osl_create(const uint64_t* keys, const uint64_t* vals, uint64_t n, int b, uint64_t seed,
                 int* err) {
    *err = 0;
    if (b < 1 || b > 4) {
        *err = -1;
        return nullptr;
    }
    for (uint64_t i = 0; i < n; ++i)
        if (keys[i] == kReservedKey) {
            *err = -1;
            return nullptr;
        }
    SkipList* s = nullptr;
    try {
        s = new SkipList();
        s->init(b, seed);
        // Stable sort of input positions by key: within equal keys the input order is
        // kept, so the last position of each run carries the winning value.
        std::vector<uint64_t> order(n);
        for (uint64_t i = 0; i < n; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](uint64_t a, uint64_t c) { return keys[a] < keys[c]; });
        Node* tail[kMaxLevels];
        for (int i = 0; i < kMaxLevels; ++i) tail[i] = s->head;
        for (uint64_t j = 0; j < n; ++j) {
            if (j + 1 < n && keys[order[j + 1]] == keys[order[j]]) continue;
            Node* x = s->new_node(keys[order[j]], vals[order[j]]);
            for (int i = 0; i < x->height; ++i) {
                tail[i]->next[i] = x;
                tail[i] = x;
            }
            ++s->count;
        }
    } catch (const std::bad_alloc&) {
        delete s;
        *err = -2;
        return nullptr;
    }
    return s;
}

// Applies the queries one at a time in arrival order and writes each query's prior
// state of its key. Returns the number of invalid queries.
uint64_t osl_execute(void* h, const uint8_t* ops, const uint64_t* keys, const uint64_t* vals,
                     uint64_t n, uint64_t* res_value, uint32_t* res_status) {
    SkipList* s = static_cast<SkipList*>(h);
    Node* update[kMaxLevels];
    uint64_t invalid = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint8_t op = ops[i];
        uint64_t key = keys[i];
        if (op > 2 || key == kReservedKey) {
            res_value[i] = 0;
            res_status[i] = O_INVALID;
            ++invalid;
            continue;
        }
        Node* x = s->find(key, update);
        res_value[i] = x ? x->value : 0;
        res_status[i] = x ? O_PRESENT : O_ABSENT;
        if (op == 1) {
            if (x)
                x->value = vals[i];
            else
                s->insert_or_assign(key, vals[i], update);
        } else if (op == 2) {
            if (x) s->unlink(x, update);
        }
    }
    return invalid;
}

uint64_t osl_size(void* h) { return static_cast<SkipList*>(h)->count; }

// Range search (Section 3.2.5), one query at a time: the live pairs with
// lo[i] <= key <= hi[i], in key order. The walk finds the last node below lo[i] top-down
// (its interception), then follows the bottom level until a key exceeds hi[i]; lo > hi
// is an empty range. Writes offsets[0..n] (query i's pairs are [offsets[i],
// offsets[i + 1]) of the output) and the first cap pairs; returns the total.
uint64_t osl_range(void* h, const uint64_t* lo, const uint64_t* hi, uint64_t n, uint64_t* offsets,
                   uint64_t* keys, uint64_t* vals, uint64_t cap) {
    SkipList* s = static_cast<SkipList*>(h);
    uint64_t total = 0;
    for (uint64_t i = 0; i < n; ++i) {
        offsets[i] = total;
        if (lo[i] > hi[i]) continue;
        Node* x = s->head;
        for (int l = s->hmax - 1; l >= 0; --l)
            while (x->next[l] && x->next[l]->key < lo[i]) x = x->next[l];
        for (Node* c = x->next[0]; c && c->key <= hi[i]; c = c->next[0]) {
            if (total < cap) {
                keys[total] = c->key;
                vals[total] = c->value;
            }
            ++total;
        }
    }
    offsets[n] = total;
    return total;
}

// Writes up to cap live pairs in key order; returns the number of live keys.
uint64_t osl_export(void* h, uint64_t* keys, uint64_t* vals, uint64_t cap) {
    SkipList* s = static_cast<SkipList*>(h);
    uint64_t k = 0;
    for (Node* x = s->head->next[0]; x; x = x->next[0], ++k) {
        if (k < cap) {
            keys[k] = x->key;
            vals[k] = x->value;
        }
    }
    return k;
}

// Highest level that holds at least one key (0 when empty).
int osl_num_levels(void* h) {
    SkipList* s = static_cast<SkipList*>(h);
    int top = 0;
    for (int i = 0; i < kMaxLevels; ++i)
        if (s->head->next[i]) top = i + 1;
    return top;
}

// Writes up to cap keys of level `level` (1 = storage layer) in order; returns its size.
uint64_t osl_export_level(void* h, int level, uint64_t* keys, uint64_t cap) {
    SkipList* s = static_cast<SkipList*>(h);
    if (level < 1 || level > kMaxLevels) return 0;
    uint64_t k = 0;
    for (Node* x = s->head->next[level - 1]; x; x = x->next[level - 1], ++k)
        if (k < cap) keys[k] = x->key;
    return k;
}

void osl_destroy(void* h) { delete static_cast<SkipList*>(h); }

}  // extern "C"
