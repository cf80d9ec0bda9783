/*
 * gf2x_gb300.h -- C ABI of libgf2x_gb300.so: constant-time multiplication of
 * dense binary polynomials (10k-60k bits and up to 131072) on an NVIDIA
 * GB300 (sm_103a), as a full product in F2[X] or reduced modulo X^n - 1.
 *
 * The operation is the one of Robert & Veron, "Faster multiplication over
 * F2[X] using AVX512 instruction set and VPCLMULQDQ instruction" (J. Crypt.
 * Eng. 2022): Sec. 2.1 states the product (two polynomials of degree at most
 * N-1, result of degree at most 2N-2, packed into 64-bit words), Sec. 1 maps
 * circulant matrix-vector products of HQC/BIKE to products in
 * F2[X]/(X^N - 1), and Sec. 2-3 (Alg. 1-3, Appendix D) give the Karatsuba
 * and Toom-3 recursions this library runs on the GPU.
 *
 * Conventions for every entry point:
 *  - Layout: a polynomial with n coefficients is ceil(n/64) little-endian
 *    uint64 limbs; coefficient k is bit (k mod 64) of limb k/64.
 *  - High bits: input bits at positions >= n are ignored; unused high bits
 *    of every output limb are written as zero.
 *  - Pointers: operand and result pointers are DEVICE pointers owned by the
 *    caller, 8-byte aligned (16-byte alignment is faster).  An output must
 *    not overlap either input (GF2X_EINVAL when the ranges overlap).
 *  - Sizes: 1 <= n <= GF2X_MAX_N, else GF2X_EUNSUPPORTED.
 *  - Asynchrony: compute calls enqueue work on `stream` (a cudaStream_t,
 *    NULL = the legacy default stream) and return at once; argument and
 *    plan errors are returned synchronously, launch errors as GF2X_ECUDA.
 *  - Constant time: no branch and no memory address of the GPU code depends
 *    on operand bits; the work done depends only on n and the plan.
 *  - Threads: a context may be used from one host thread at a time.
 *  - No C++ exception crosses this interface.
 */
#ifndef GF2X_GB300_H
#define GF2X_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GF2X_OK = 0,
    GF2X_EINVAL = 1,        /* bad pointer, overlap, bad flag or bad plan spec */
    GF2X_ENOMEM = 2,        /* an allocation failed, or a fixed workspace is too small */
    GF2X_ECUDA = 3,         /* a CUDA runtime call failed */
    GF2X_ETIMEOUT = 4,      /* a bounded wait ran out */
    GF2X_EUNSUPPORTED = 5,  /* n outside [1, GF2X_MAX_N] or a plan that does not fit */
    GF2X_EBUSY = 6,         /* resource in use (e.g. admission refused) */
    GF2X_EDEVICE = 7        /* the checked-mode kernel reported a broken invariant */
} gf2x_status;

#define GF2X_MAX_N 131072u
#define GF2X_MAX_LEVELS 8

/* Level kinds of a recursion plan. */
#define GF2X_LEVEL_KARATSUBA 0u  /* k-way Karatsuba split, k in {2,3,5}: Alg. 1 (KaratRec), Alg. 2 (Karat3), Alg. 3 (Karat5) */
#define GF2X_LEVEL_TOOM3 1u      /* word-aligned Toom-3 at 0, 1, x, x+1, inf with x = X^w: Sec. 3.2 and Appendix D */

/* Per-item / call flags. */
#define GF2X_REDUCE 1u           /* result is a*b mod X^n - 1 (ceil(n/64) limbs), else the full product */

/* Batch flags. */
#define GF2X_BATCH_PERSISTENT 1u  /* grid of (SMs x resident CTAs); each CTA loops over the items */
#define GF2X_BATCH_ITEMS_ON_DEVICE 2u /* `items` points to device memory (gf2x_item array) */
#define GF2X_BATCH_LARGEST_FIRST 4u   /* order items by decreasing n (sizes are public) before the launch */
#define GF2X_BATCH_SHARED_A 8u        /* gf2x_mul_strided: one a for every product (a fixed key polynomial) */
#define GF2X_BATCH_DYNAMIC 16u        /* gf2x_mul_batched, persistent: CTAs take items in order from a counter */

/*
 * A recursion plan: `nlev` split levels from the top down, then a leaf of
 * `leaf_words` 32-bit words multiplied by a constant-time carry-less
 * schoolbook.  Sizes follow Sec. 3.2: a Karatsuba level of child size E has
 * parent size k*E; a Toom-3 level with word shift W (w = 32W bits) and child
 * size E has parent size 3(E - 2W).  The top size must cover ceil(n/32)
 * words; leaf_words = 0 picks the smallest compiled leaf that does.
 *   kind[l]: GF2X_LEVEL_KARATSUBA (arg[l] = k) or GF2X_LEVEL_TOOM3 (arg[l] = W).
 *   threads: CTA size (0 = chosen from the leaf count).
 *   seq_top: 1 = the CTA multiplies the top level's children one after the
 *            other (less shared memory, for the largest sizes).
 *   fuse_leaf: 1 = the last level (a 2-way Karatsuba) runs inside the leaf
 *            thread, in registers (leaf_words <= 10); 0 = it runs as a
 *            shared-memory level like the others.
 *   split_top: 1 = the top level runs across CTAs: one kernel evaluates the
 *            children into global scratch, the children are multiplied as
 *            independent products (levels 1.. of the plan, where seq_top then
 *            applies), and one kernel interpolates; for sizes whose whole tree
 *            does not fit one CTA's shared memory (up to GF2X_MAX_N).  The
 *            child size must be an even number of words.
 */
typedef struct {
    uint32_t nlev;
    uint32_t kind[GF2X_MAX_LEVELS];
    uint32_t arg[GF2X_MAX_LEVELS];
    uint32_t leaf_words;
    uint32_t threads;
    uint32_t seq_top;
    uint32_t fuse_leaf;
    uint32_t split_top;
} gf2x_plan_spec;

/* Facts about a plan for one n (host-side only, needs no GPU). */
typedef struct {
    uint32_t n;
    uint32_t top_words;          /* padded operand size, 32-bit words */
    uint32_t leaf_words;
    uint32_t nleaves;            /* leaf products per multiplication */
    uint32_t threads;
    uint32_t smem_bytes;         /* dynamic shared memory per CTA */
    uint32_t level_words[GF2X_MAX_LEVELS + 1]; /* operand size at each depth (top first, leaf last) */
    uint64_t ops_full;           /* modelled 32-bit integer operations per full product */
    uint64_t ops_leaf;           /* of which in the leaf schoolbook */
    uint64_t clmul64;            /* 64x64-bit word products (the Karatsuba-variants complexity table of Sec. 2.1); leaf_words even */
    uint64_t bytes_in;           /* HBM bytes read per product */
    uint64_t bytes_out_full;     /* HBM bytes written, full product */
    uint64_t bytes_out_reduced;  /* HBM bytes written, reduced product */
    uint64_t scratch_bytes;      /* global scratch per product (split plans; 0 otherwise) */
} gf2x_plan_info;

/* Item of a batched call.  Pointers as in the conventions above. */
typedef struct {
    const uint64_t *a;
    const uint64_t *b;
    uint64_t *out;
    uint32_t n;
    uint32_t flags;              /* GF2X_REDUCE or 0 */
} gf2x_item;

/* One row copy of gf2x_copy_rows (device pointers, 8-byte aligned). */
typedef struct {
    const uint64_t *src;
    uint64_t *dst;
    uint64_t limbs;              /* 0: an empty entry (padding) */
} gf2x_copy_row;

typedef struct gf2x_ctx gf2x_ctx;
typedef void *gf2x_stream;       /* cudaStream_t */

/* Human-readable name of a status code (static storage). */
const char *gf2x_status_str(gf2x_status s);

/* Library version string, e.g. "gf2x_gb300 1.0 sm_103a". */
const char *gf2x_version(void);

/* Default plan spec for size n (what a fresh context uses).  Host only. */
gf2x_status gf2x_default_spec(uint32_t n, gf2x_plan_spec *spec);

/* Validate `spec` for size n and describe it.  Host only, needs no GPU.
 * GF2X_EINVAL for a malformed spec, GF2X_EUNSUPPORTED if it does not cover
 * n or does not fit in one CTA's shared memory. */
gf2x_status gf2x_plan_info_get(uint32_t n, const gf2x_plan_spec *spec, gf2x_plan_info *info);

/* Parse a plan spec from text "T2.K3.K2.K2/8/288/0/1/0" (levels / leaf_words /
 * threads / seq_top / fuse_leaf / split_top; the last five fields optional,
 * 0 = automatic or off). */
gf2x_status gf2x_spec_parse(const char *text, gf2x_plan_spec *spec);

/* Create a context on CUDA device `device` (made current on the calling
 * thread).  The context owns device-side plan tables, item staging buffers
 * and scratch.
 *  - workspace_bytes = 0: scratch grows on demand -- the split-plan scratch,
 *    the unbalanced/Toom scratch, the host-buffer pipeline and the item
 *    staging are allocated (cudaMalloc / cudaMallocHost, which synchronize)
 *    by the first compute call that needs more.
 *  - workspace_bytes > 0: one device arena of that size (rounded down to
 *    1 KiB) is allocated here -- half split-plan scratch, a quarter
 *    unbalanced/Toom scratch, a quarter host-buffer pipeline -- with 4 x
 *    16384 item staging slots, and NO compute call allocates afterwards:
 *    batches run in chunks that fit, host item batches above 16384 items run
 *    in pieces (each piece ordered and grouped by itself), and a call whose
 *    single product does not fit returns GF2X_ENOMEM.
 *  - plan_db_path: a plan database to install (see gf2x_ctx_load_plan_db;
 *    the batch bucket nearest to 4096 is used), or NULL for default plans.
 * Errors: GF2X_ENOMEM when an allocation fails, GF2X_ECUDA for another CUDA
 * failure, the plan database's status when it is rejected (no context is
 * returned then). */
gf2x_status gf2x_ctx_create(gf2x_ctx **ctx, int device, size_t workspace_bytes, const char *plan_db_path);

/* Allocations the context has made since it was created (cudaMalloc and
 * cudaMallocHost calls, creation included) and their bytes; either pointer
 * may be NULL.  With a fixed workspace the count stays at its value after
 * gf2x_ctx_create.  Host only. */
gf2x_status gf2x_ctx_alloc_count(gf2x_ctx *ctx, uint64_t *allocations, uint64_t *bytes);

/* For tests of the GF2X_ENOMEM paths: the next `count` device or pinned
 * allocations of any context fail as if the memory were exhausted (no CUDA
 * call is made for them).  Returns the previous count.  Process-wide. */
uint32_t gf2x_debug_fail_next_allocs(uint32_t count);

/* Release everything the context owns (waits for its work to finish). */
void gf2x_ctx_destroy(gf2x_ctx *ctx);

/* Use `spec` for every later product of size n in this context
 * (spec = NULL restores the default).  Host-side validation only.  On an
 * error (a spec that does not fit n, or GF2X_EUNSUPPORTED "plan table full"
 * after 8192 distinct plans in one context) the previous plan stays in force. */
gf2x_status gf2x_ctx_set_plan(gf2x_ctx *ctx, uint32_t n, const gf2x_plan_spec *spec);

/* Load a plan database written by the autotuner: text lines
 * "n batch_bucket spec", '#' comments.  For each n the entry whose batch
 * bucket is nearest (in log2) to batch_hint becomes the context's plan.
 * GF2X_EINVAL if the file cannot be read or an entry is rejected (the
 * valid entries are still installed). */
gf2x_status gf2x_ctx_load_plan_db(gf2x_ctx *ctx, const char *path, size_t batch_hint);

/* The spec the context currently uses for size n. */
gf2x_status gf2x_ctx_get_plan(gf2x_ctx *ctx, uint32_t n, gf2x_plan_spec *spec);

/* Enable (1) or disable (0) the checked kernels: they verify on the GPU the
 * exactness of every division by x and x+1 and the zero padding, and record
 * a violation for gf2x_ctx_sync_status.  Off by default. */
gf2x_status gf2x_ctx_set_checked(gf2x_ctx *ctx, int on);

/* Full product c = a*b in F2[X]: a, b have ceil(n/64) limbs, c gets
 * ceil((2n-1)/64) limbs.  One launch of one CTA (Sec. 2.1). */
gf2x_status gf2x_mul(gf2x_ctx *ctx, uint64_t *c, const uint64_t *a, const uint64_t *b,
                     uint32_t n, gf2x_stream stream);

/* Reduced product r = a*b mod (X^n - 1): r gets ceil(n/64) limbs
 * (the circulant product of Sec. 1).  One launch of one CTA. */
gf2x_status gf2x_mulmod_xn1(gf2x_ctx *ctx, uint64_t *r, const uint64_t *a, const uint64_t *b,
                            uint32_t n, gf2x_stream stream);

/* `count` independent products of one size n in one launch.  Operand p is
 * a + p*stride_in, result p is out + p*stride_out (strides in limbs, at
 * least ceil(n/64) and the output size).  flags: GF2X_REDUCE; batch_flags:
 * GF2X_BATCH_PERSISTENT (a grid of SMs x resident CTAs that take the
 * products in order from a device counter of the context, zeroed by a
 * memset on `stream`; with a split plan, its child products are taken
 * from such a counter; without the flag, one CTA per product (per child),
 * which measured faster on GB300 when the batch is not a multiple of the
 * grid, e.g. 7.93 against 7.73 M products/s at 4096 x 17669), and
 * GF2X_BATCH_SHARED_A, with which every product
 * reads the same a (its ceil(n/64) limbs; only b advances by stride_in),
 * as when one public-key polynomial of the HQC/BIKE operations of Sec. 1
 * serves many encapsulations.  The results are those of the unshared call
 * with a copied into every row; the saving is a's reads from memory (a
 * stays in L2), not arithmetic. */
gf2x_status gf2x_mul_strided(gf2x_ctx *ctx, uint64_t *out, const uint64_t *a, const uint64_t *b,
                             uint32_t n, size_t count, size_t stride_in, size_t stride_out,
                             uint32_t flags, uint32_t batch_flags, gf2x_stream stream);

/* `count` independent products of possibly different sizes.
 *  - Host `items`: every item is checked, its plan resolved, and the array
 *    copied through a pinned staging buffer of the context (a ring of four;
 *    a reused buffer is first waited for on the host).  Items whose plans
 *    share a leaf size run in one launch (one launch per leaf size); items
 *    with a split plan run as that plan's three launches per plan.
 *  - GF2X_BATCH_ITEMS_ON_DEVICE: `items` is a device array of gf2x_item read
 *    by the kernel, which looks each plan up by n on the device among the
 *    sizes of the last gf2x_ctx_prepare call; those plans must share one
 *    leaf size and none may be a split plan (else GF2X_EUNSUPPORTED).  The
 *    launch gets the largest CTA and
 *    shared memory of those plans; a plan that does not match the launch is
 *    refused on the device and reported (never run).  An item whose n has no
 *    plan is skipped and reported by gf2x_ctx_sync_status; an item with
 *    n = 0 is an empty slot, skipped silently (padding for fixed-size
 *    captured launches).  Nothing is
 *    checked on the host and nothing is copied, so the call can be captured
 *    in a CUDA graph; the array must stay valid until the work completes.
 *  - GF2X_BATCH_PERSISTENT: a grid of (SMs x resident CTAs), each CTA
 *    looping over items i, i + grid, i + 2 grid, ...; otherwise one CTA per
 *    item.  Items of uneven sizes balance best ordered largest first (every
 *    CTA then draws one item of each size band per round).
 *  - GF2X_BATCH_LARGEST_FIRST (host items): larger n first.
 *  - GF2X_BATCH_DYNAMIC (with GF2X_BATCH_PERSISTENT): each CTA takes its
 *    next item from a device counter of the context (zeroed by a memset on
 *    `stream` before the launch, which a CUDA graph captures as well), so
 *    items are started in array order as CTAs free up -- with items sorted
 *    largest first this is longest-processing-time-first scheduling.
 *    Outside a stream capture the context's 256 counters are used round
 *    robin, and a counter's next launch first waits (on its stream) for the
 *    event recorded behind its previous launch, whatever stream that was
 *    on.  A captured launch keeps a counter of its own for the graph's
 *    lifetime (1024 per context; beyond that, captured launches take items
 *    in the static order i, i + grid, ...).  Replays of one graph must not
 *    overlap each other. */
gf2x_status gf2x_mul_batched(gf2x_ctx *ctx, const gf2x_item *items, size_t count,
                             uint32_t batch_flags, gf2x_stream stream);

/* The products of gf2x_mul_strided with operands and results in HOST memory
 * (the operation of Sec. 1; the paper's CPU code has no host/device split,
 * so this call has no counterpart there).  a, b, out: host arrays, same
 * layout, strides and flags as gf2x_mul_strided; page-locked memory lets
 * the copies overlap the products (pageable memory works, with copies that
 * do not overlap).  The batch runs in up to four chunks through two sets of
 * device buffers owned by the context: while one chunk is multiplied (one
 * CTA per product, on one of two compute streams of the context, one per
 * buffer set, so that a chunk's launch can fill the SMs the other's last
 * wave leaves idle), the next chunk's operands are copied in and the
 * previous chunk's results copied out, on two copy streams of the context,
 * all ordered by events.
 *  - Ordering: without GF2X_HOST_INPUTS_READY the operand copies wait for
 *    all work already enqueued on `stream`, and the products and result
 *    copies wait for the operand copies, so the whole call follows that
 *    work.  With GF2X_HOST_INPUTS_READY nothing of the call waits for
 *    `stream`: a and b must be final and `out` unused by earlier work at
 *    the call, and the copies and products may overlap that work (e.g. the
 *    previous call's last products).  A device buffer set is reused only
 *    after its previous product and result copy, whichever call (and
 *    stream) made them.  `stream` waits for the last result copy:
 *    synchronize it before reading `out`; the caller must not change a or
 *    b, nor read out, until then.
 *  - Rows: only the ceil(n/64) operand limbs of each row are read and only
 *    the result limbs written; limbs between rows (strides above the sizes)
 *    are left untouched.
 *  - Memory: the device buffers grow to 2 x (chunk products) x (2 ceil(n/64)
 *    + result limbs) limbs on the first call that needs more (cudaMalloc,
 *    which synchronizes the device) and are kept until gf2x_ctx_destroy.
 *  - Errors: as gf2x_mul_strided (GF2X_EINVAL for null or overlapping host
 *    ranges, bad strides or flags); after a GF2X_ECUDA the results are
 *    undefined. */
#define GF2X_HOST_INPUTS_READY (1u << 8)

gf2x_status gf2x_mul_strided_host(gf2x_ctx *ctx, uint64_t *out, const uint64_t *a, const uint64_t *b,
                                  uint32_t n, size_t count, size_t stride_in, size_t stride_out,
                                  uint32_t flags, gf2x_stream stream);

/* `count` full products of operands of different sizes: row p of a (na
 * bits in ceil(na/64) limbs, stride_a limbs apart) times row p of b (nb
 * bits, stride_b), result row p of ceil((na + nb - 1)/64) limbs at out +
 * p*stride_out.  Bits above na / nb in the operands' top limbs are ignored.
 * With nb <= na (else the operands swap roles; the product commutes) the
 * call runs either one equal-size product of the zero-extended operands
 * (the padding of Sec. 3.2) or, when the context's plans model it cheaper,
 * k = ceil(na/m) products of a's m-bit chunks times b, m = 64 ceil(nb/64),
 * added at offsets i m (the one-sided split of Sec. 2.1):
 * a padding kernel, the batched products, an overlap-add kernel, all on
 * `stream`.  Without a plan of its own for m, the chunk products run under
 * the spec of nb's plan where it covers m (same limb count; the context's
 * plan for m is left unset).  Scratch: a device buffer of the context, grown on demand
 * (cudaMalloc, which synchronizes the device) up to 256 MiB per group of
 * products (larger batches run in groups) and kept until
 * gf2x_ctx_destroy; calls on different streams are ordered through it.
 * Errors: GF2X_EUNSUPPORTED for a size outside [1, 131072]; GF2X_EINVAL for
 * null or misaligned pointers, short strides, results overlapping an
 * operand. */
gf2x_status gf2x_mul_unbalanced(gf2x_ctx *ctx, uint64_t *out, const uint64_t *a, uint32_t na, size_t stride_a,
                                const uint64_t *b, uint32_t nb, size_t stride_b, size_t count, size_t stride_out,
                                gf2x_stream stream);

/* Constant-time products of a dense a and a sparse b mod X^n - 1, the
 * operand shape of the HQC/BIKE operations of Sec. 1 (a public dense
 * polynomial times a secret low-weight one).  b = sum_j X^(pos[j]) over its w
 * positions (repeated positions cancel, as in F2); result row p = a_p * b_p
 * mod X^n - 1 in ceil(n/64) limbs, bits above n zero.  Sec. 1 rules out
 * multiplications that use the sparsity through branches or memory
 * addresses; this one never does: each position becomes the select masks of
 * barrel shifters (register renames and fixed-offset lane shuffles, every
 * stage executed) and the count of a funnel shift on the doubled vector
 * a + X^n a, so the work, the addresses and the shuffle lanes depend on n,
 * w and count only.
 *  - a: count rows of ceil(n/64) limbs, stride_a limbs apart (bits above n
 *    ignored); pos: count rows of w uint32 positions, stride_pos entries
 *    apart, each < n (a position >= n gives an unspecified row, never an
 *    access outside the operands); r: count rows, stride_r limbs apart.
 *  - One CTA per product (its four warps share the positions), one launch
 *    on `stream`; n up to 65536.
 *  - Errors: GF2X_EUNSUPPORTED for n outside [1, 65536]; GF2X_EINVAL for
 *    null or misaligned pointers (8 bytes for a and r, 4 for pos), short
 *    strides, results overlapping a or pos. */
gf2x_status gf2x_mulmod_sparse(gf2x_ctx *ctx, uint64_t *r, const uint64_t *a, const uint32_t *pos, uint32_t w,
                               uint32_t n, size_t count, size_t stride_a, size_t stride_pos, size_t stride_r,
                               gf2x_stream stream);

/* `count` products of one size n through a Toom-4 top level (Toom-Cook
 * 4-7, the next member of Sec. 3's Toom-Cook family after Toom-3; in the
 * size ranges of gf2x listed in the Toom-Cook complexity table of Sec. 3.1
 * it takes over from Toom-3 above degree 22143, after a band of sizes where
 * the two cost about the same).  Same
 * operands, strides, flags (GF2X_REDUCE) and results as gf2x_mul_strided.
 * Each operand is cut into four parts of m = ceil(ceil(n/32)/4) 32-bit
 * words and evaluated at 0, 1, x, x+1, x^2, x^2+1 and inf with x = X^32
 * (an evaluation kernel); the seven products of E = m + 6 (rounded up to
 * even) words run as one batch under the context's plan for 32 E bits;
 * an interpolation kernel (exact divisions by x, x+1 and x^2+x+1 as word
 * shifts and prefix XORs) recomposes, and folds mod X^n - 1 on request.
 * Scratch: the context buffer of gf2x_mul_unbalanced (112 E bytes per
 * product, groups of at most 256 MiB).  Errors: as gf2x_mul_strided. */
gf2x_status gf2x_mul_toom4(gf2x_ctx *ctx, uint64_t *out, const uint64_t *a, const uint64_t *b, uint32_t n,
                           size_t count, size_t stride_in, size_t stride_out, uint32_t flags, gf2x_stream stream);

/* The same through a Toom-5 top level (Toom-Cook 5-9, the next range of
 * the Toom-Cook complexity table of Sec. 3.1): five parts of
 * m = ceil(ceil(n/32)/5) words, nine points (those of gf2x_mul_toom4 plus x^2+x and x^2+x+1, whose
 * differences again factor into x, x+1 and x^2+x+1), nine child products of
 * E = m + 8 (even) words; scratch 144 E bytes per product. */
gf2x_status gf2x_mul_toom5(gf2x_ctx *ctx, uint64_t *out, const uint64_t *a, const uint64_t *b, uint32_t n,
                           size_t count, size_t stride_in, size_t stride_out, uint32_t flags, gf2x_stream stream);

/* Products r_j = a * b_j mod X^n - 1 of ONE polynomial a with `count`
 * polynomials b_j on the tensor cores: the circulant matrix of a (Sec. 1)
 * times the matrix of the b_j as an integer GEMM in block-scaled fp4
 * (tcgen05.mma kind::mxf4, operands 0/1, every scale 1.0, exact fp32 counts
 * in tensor memory), the product bits being the counts' parities.  For the
 * operand shape of Sec. 1 where one public polynomial (an HQC/BIKE key)
 * multiplies many vectors; results equal gf2x_mul_strided with
 * GF2X_BATCH_SHARED_A and GF2X_REDUCE, bit for bit.
 *  - a: ceil(n/64) limbs; b: count rows, stride_b limbs apart; r: count
 *    rows of ceil(n/64) limbs, stride_r limbs apart (bits above n ignored in
 *    the operands, zero in the results).
 *  - n odd, 1 <= n <= 65535 (the HQC and BIKE moduli are primes), else
 *    GF2X_EUNSUPPORTED.  The work is n^2 multiply-adds per product, so the
 *    call pays at the smaller sizes; the Karatsuba/Toom path wins again as n
 *    grows.
 *  - Launches on `stream`: the sequence of a, then per group of products an
 *    unpacking kernel, the GEMM (persistent, one CTA per SM, all of its
 *    tensor memory) and a reordering kernel.  Scratch: the context buffer of
 *    gf2x_mul_unbalanced, about (count/128) ceil(n/64) 4 KiB + count n/8
 *    bytes plus 8 n bytes for a.  A kernel wait that runs out (none is
 *    expected) is reported by gf2x_ctx_sync_status as GF2X_ETIMEOUT.
 *  - Constant time: addresses and branches depend on n and count only.
 *  - Errors: GF2X_EINVAL for null or misaligned pointers, short strides,
 *    results overlapping a or b; GF2X_ENOMEM when the scratch cannot hold a
 *    group of 128 products. */
gf2x_status gf2x_mulmod_shared_tc(gf2x_ctx *ctx, uint64_t *r, const uint64_t *a, const uint64_t *b, uint32_t n,
                                  size_t count, size_t stride_b, size_t stride_r, gf2x_stream stream);

/* The kernel shape gf2x_mulmod_sparse uses for n (host only, needs no GPU).
 * A warp holds words_per_lane registers of the doubled vector, word
 * lane + 32 k in register k, and result_words_per_lane accumulator
 * registers (32 x result_words_per_lane >= ceil(n/32) + 1).  The word offset
 * of a position is applied by shared_stages shifts in shared memory (its top
 * bits, each shift >= 256 words), register_stages shifts by whole registers
 * and lane_stages (5) lane rotations; its bit offset by a funnel shift.
 * GF2X_EUNSUPPORTED for n outside [1, 65536]. */
typedef struct {
    uint32_t n;
    uint32_t words_per_lane;
    uint32_t result_words_per_lane;
    uint32_t shared_stages;
    uint32_t register_stages;
    uint32_t lane_stages;
    uint32_t smem_bytes;            /* dynamic shared memory per CTA (four warps) */
} gf2x_sparse_info;

gf2x_status gf2x_sparse_info_get(uint32_t n, gf2x_sparse_info *info);

/* Build and upload (synchronously on `stream`) the current plans of the
 * given sizes, so that later calls and CUDA graph captures find them ready,
 * and make exactly these sizes the ones device-item batches accept (their
 * plans are looked up by n on the device; other sizes are reported as
 * having no plan). */
gf2x_status gf2x_ctx_prepare(gf2x_ctx *ctx, const uint32_t *sizes, size_t count, gf2x_stream stream);

/* Launch shape the context uses for size n: CTA threads, dynamic shared
 * memory, resident CTAs per SM and the SM count (any pointer may be NULL). */
gf2x_status gf2x_ctx_launch_shape(gf2x_ctx *ctx, uint32_t n, uint32_t *threads, uint32_t *smem_bytes,
                                  uint32_t *blocks_per_sm, uint32_t *sm_count);

/* `count` row copies in one launch on `stream`: entry i of the DEVICE array
 * `rows` copies rows[i].limbs 64-bit words from rows[i].src to rows[i].dst
 * (ranges must not overlap; entries with limbs = 0 are skipped).  Nothing is
 * checked or copied on the host, so the call can be captured in a CUDA
 * graph.  The paper has no counterpart: the serving loop uses it to stage
 * the operands of the requests it admits into its device-memory budget. */
gf2x_status gf2x_copy_rows(gf2x_ctx *ctx, const gf2x_copy_row *rows, size_t count, gf2x_stream stream);

/* Wait for `stream`, then report and clear any checked-mode violation
 * (GF2X_EDEVICE) or asynchronous CUDA error (GF2X_ECUDA). */
gf2x_status gf2x_ctx_sync_status(gf2x_ctx *ctx, gf2x_stream stream);

/* gf2x_ctx_sync_status with a deadline: polls the stream every 50 us (no
 * blocking synchronize) for at most timeout_ms; GF2X_ETIMEOUT if its work
 * has not finished by then (the work goes on; wait again or destroy the
 * context, which waits), else the result of gf2x_ctx_sync_status. */
gf2x_status gf2x_ctx_wait(gf2x_ctx *ctx, gf2x_stream stream, uint32_t timeout_ms);

/* Text of the last error recorded in the context (static until the next
 * call on it). */
const char *gf2x_ctx_last_error(gf2x_ctx *ctx);

/* ---- Products with no allocation at all ----------------------------------
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot call cudaMalloc: a host program whose framework owns all device
 * memory through its own allocator (memory taken behind its back breaks its
 * accounting), a service that reserves its whole memory budget at start-up
 * and must not grow afterwards, and code that must not stall other streams
 * (cudaMalloc and cudaFree may synchronize the device).  Such callers can
 * hand the library their operand and result buffers, but no scratch.
 *
 * gf2x_mul_strided_static computes the same `count` products as
 * gf2x_mul_strided (same operand/result layout, strides in limbs, flags
 * GF2X_REDUCE or 0), with a split plan (spec->split_top = 1; spec = NULL
 * picks the split plan with the fewest modelled operations for n), and needs
 * no context.  Its scratch is a file-scope device array of
 * GF2X_STATIC_SCRATCH_BYTES that every GPU which loads the library holds
 * until the process exits; its two plans live in a second such array,
 * written by a one-block kernel that receives them as launch parameters.
 * It calls no cudaMalloc, cudaFree or other allocating routine.
 *  - Set-up: the first call on a device (with that device current) looks up
 *    the arrays' device addresses (cudaGetSymbolAddress) and sets the
 *    kernels' shared-memory limits; make that first call before any stream
 *    capture.
 *  - Limit: count x gf2x_plan_info.scratch_bytes of the plan must not exceed
 *    GF2X_STATIC_SCRATCH_BYTES, else GF2X_EUNSUPPORTED (split the batch).
 *  - Sharing: every call uses the same arrays, which keep the last call's
 *    contents (nothing in them needs to start at zero: every word of the
 *    scratch is written before it is read); calls whose work overlaps on the
 *    GPU (other streams, other host threads) race -- order them on one
 *    stream.
 *  - Errors: GF2X_EINVAL for bad pointers, overlap, flags or a spec that is
 *    not a split plan; launch failures as GF2X_ECUDA.  There is no context
 *    and so no error word: the kernels' own refusal of a plan that does not
 *    match their launch is not reported, and cannot arise here, because the
 *    plans are built on the host for this very launch. */
#define GF2X_STATIC_SCRATCH_BYTES (4u << 20)

gf2x_status gf2x_mul_strided_static(uint64_t *out, const uint64_t *a, const uint64_t *b, uint32_t n, size_t count,
                                    size_t stride_in, size_t stride_out, uint32_t flags,
                                    const gf2x_plan_spec *spec, gf2x_stream stream);

/* ---- Plan cost model network (the autotuner's learned part) -------------
 * A two-layer perceptron y = w2 . relu(W1 x + b1) + b2 in fp32 that predicts
 * the log time of a recursion plan from its descriptor.  The paper has no
 * counterpart: it chooses constructions per degree by measurement (Sec. 3,
 * the Toom-3 timing tables of Sec. 3.2 and 3.3); the network only orders the
 * candidates the autotuner measures.  All pointers are device pointers; the
 * parameter vector is W1 [hidden x in_dim] row-major, b1 [hidden],
 * w2 [hidden], b2 [1] (gf2x_mlp_param_count floats).  1 <= in_dim <= 64,
 * 1 <= hidden <= 128, else GF2X_EINVAL.  Asynchronous on `stream`. */

/* Number of fp32 parameters of the network. */
size_t gf2x_mlp_param_count(int in_dim, int hidden);

/* y[s] = network(x[s]) for s < batch; x is [batch x in_dim] row-major. */
gf2x_status gf2x_mlp_forward(const float *params, const float *x, float *y, int batch, int in_dim, int hidden,
                             gf2x_stream stream);

/* Gradient of L = (1/batch) sum_s (y_s - target_s)^2 with respect to the
 * parameters into grad (overwritten), and L into *loss (device float). */
gf2x_status gf2x_mlp_grad(const float *params, const float *x, const float *target, float *grad, float *loss,
                          int batch, int in_dim, int hidden, gf2x_stream stream);

/* One Adam step (Kingma & Ba, with bias correction for step >= 1) on
 * params using grad and the moment buffers m, v (nparams floats each). */
gf2x_status gf2x_mlp_adam(float *params, const float *grad, float *m, float *v, size_t nparams, float lr,
                          float beta1, float beta2, float eps, int step, gf2x_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GF2X_GB300_H */
