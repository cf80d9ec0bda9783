// plan.h -- the recursion plan as the GPU kernels read it (POD, shared by
// host and device code).
//
// A plan splits a product of two T0-word operands (32-bit words) through
// `nlev` levels down to leaves of S words:
//   Karatsuba k-way (Alg. 1 k=2, Alg. 2 k=3, Alg. 3 k=5): parent T = k E,
//     children = k singles then the k(k-1)/2 pair sums, in lexicographic
//     order; reconstruction term p (0 <= p <= 2k-2, at word offset pE) is the
//     XOR of the singles i and the pairs (i,j), i<j, with i+j = p, plus every
//     single i with 0 <= p-i < k (this is Alg. 1-3 written for any k);
//   Toom-3 with x = X^w, w = 32 W bits (Sec. 3.2, Appendix D): parent T = 3n',
//     five children of E = n' + 2W words at the points 0, 1, x, x+1, inf.
// Every node's operands sit in one slot of 2*size words (A then B); the
// node's product later overwrites the same slot.
#pragma once
#include <stdint.h>

namespace gf2x {

constexpr int kMaxLevels = 8;
constexpr int kMaxTerms = 8;

enum : uint32_t { kKaratsuba = 0, kToom3 = 1 };

// x / d for x * d < 2^32 (host-checked): q = umulhi(x, m), m = floor(2^32/d) + 1.
struct FastDiv {
    uint32_t d;
    uint32_t m;
};

struct GLevel {
    uint32_t kind;      // kKaratsuba or kToom3
    uint32_t k;         // split count (Toom-3: 3)
    uint32_t W;         // Toom-3 shift in words (Karatsuba: 0)
    uint32_t T;         // parent operand words
    uint32_t E;         // child operand words
    uint32_t np;        // Toom-3 part words n' = E - 2W (Karatsuba: E)
    uint32_t nch;       // children per parent
    uint32_t npar;      // parents at this level handled in one pass
    uint32_t in_off;    // shared-memory word offset of the parent slots
    uint32_t ch_off;    // shared-memory word offset of the children slots
    FastDiv div2E, divnch, divE, div2T, divhE;
    uint8_t sel[16][2];                 // Karatsuba child j = X[sel0] ^ X[sel1] (sel1 = 255: single)
    uint8_t nterms[2 * 5 - 1];
    uint8_t terms[2 * 5 - 1][kMaxTerms];  // children XORed into reconstruction term p
    uint8_t pair;       // 1: this 2-way level and the next run as one pass (9 grandchildren);
                        // 2: the second level of such a pair (no pass of its own)
    uint8_t pad_[2];
};

struct GPlan {
    uint32_t n;          // coefficients
    uint32_t L32;        // ceil(n/32)
    uint32_t L64;        // ceil(n/64)
    uint32_t Lfull64;    // ceil((2n-1)/64)
    uint32_t T0;         // top operand words
    uint32_t nlev;
    uint32_t S;          // leaf words
    uint32_t nleaf_pass; // leaves multiplied per leaf pass
    uint32_t seq_top;    // 1: top level's children one at a time
    uint32_t threads;
    uint32_t smem_words; // dynamic shared memory, 32-bit words
    uint32_t top_off;    // slot of the top operands / product
    uint32_t prod_off;   // seq_top: the top level's children products
    uint32_t tmp_off;    // Toom-3 interpolation temporaries
    uint32_t part_off;   // prefix-XOR scan partials
    uint32_t part_words;
    uint32_t checked;    // verify exactness invariants on the device
    uint32_t fuse_k2;    // 1: the last level is a 2-way Karatsuba done inside the leaf thread
    uint32_t split;      // 1: this is the top level of a split plan (children go through global scratch)
    uint32_t pad2_;
    GLevel lev[kMaxLevels];
};

// One product handed to a kernel.
struct DevItem {
    const uint64_t *a;
    const uint64_t *b;
    uint64_t *out;
    uint32_t plan;       // index into the plan table
    uint32_t flags;      // bit 0: reduce mod X^n - 1
};

// How a launch finds its items.
struct LaunchArgs {
    const GPlan *plans;       // device plan table
    const DevItem *items;     // mode kItemsArray
    DevItem base;             // mode kItemsSingle / kItemsStrided
    uint64_t stride_in;       // limbs, mode kItemsStrided
    uint64_t stride_out;
    uint32_t count;
    uint32_t mode;
    uint32_t persistent;
    uint32_t shared_a;        // mode kItemsStrided: 1 = every product reads the same a
    uint32_t *err;            // device error word (checked mode), may be null
    const uint32_t *plan_of_n; // mode kItemsUser: plan slot of every n (kNoPlan if none)
    uint32_t *work_counter;   // non-null: persistent CTAs take items in order from this counter (zeroed before the launch)
};

// kItemsUser: the items are the caller's gf2x_item array on the device, whose
// fourth field is n instead of a plan slot.
enum : uint32_t { kItemsSingle = 0, kItemsArray = 1, kItemsStrided = 2, kItemsUser = 3 };
constexpr uint32_t kNoPlan = 0xffffffffu;
constexpr uint32_t kEmptyItem = 0xfffffffeu;  // device item with n = 0: a padding slot, skipped

// Checked-mode error codes (bit flags, OR-ed into *err).
enum : uint32_t { kErrDivX = 1, kErrDivX1 = 2, kErrPad = 4, kErrNoPlan = 8, kErrPlanMismatch = 16, kErrDivX2X1 = 32,
                 kErrTimeout = 64 };   // kErrTimeout: a bounded wait in a kernel ran out

}  // namespace gf2x
