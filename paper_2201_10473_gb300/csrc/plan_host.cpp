// plan_host.cpp -- host-side plan algebra: sizes, shared-memory layout,
// operation model and the default plan choice.  Needs no GPU.
//
// Size rule (Sec. 3.2): a Toom-3 level whose children have E words has
// parts of n' = E - 2W words and a parent of t = 3n' words ("n + 2w/64 is
// the size of the elementary multiplication"); a k-way Karatsuba level has
// parent k*E (Sec. 2.1, t = 2^r, 3*2^r, 5*2^r words).  Working in 32-bit
// words, the paper's 64-bit sizes are the even cases.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gf2x_gb300.h"
#include "plan.h"
#include "plan_host.h"

namespace gf2x {

const uint32_t kLeafSizes[kNumLeafSizes] = {4, 6, 8, 10, 12, 16};

uint32_t max_threads_for_leaf(uint32_t S) { return S <= 6 ? 768u : 512u; }

bool leaf_supported(uint32_t S)
{
    for (uint32_t s : kLeafSizes)
        if (s == S)
            return true;
    return false;
}

static FastDiv make_div(uint32_t d)
{
    FastDiv f;
    f.d = d;
    f.m = d <= 1 ? 0u : (uint32_t)((1ull << 32) / d + 1ull);
    return f;
}

static uint32_t round_up(uint32_t x, uint32_t m) { return (x + m - 1) / m * m; }

// Level sizes bottom-up from the leaf; false if a Toom part would be empty.
static bool level_sizes(const gf2x_plan_spec &s, uint32_t S, uint32_t *sz)
{
    sz[s.nlev] = S;
    for (int l = (int)s.nlev - 1; l >= 0; --l) {
        uint64_t E = sz[l + 1];
        uint64_t T;
        if (s.kind[l] == GF2X_LEVEL_KARATSUBA) {
            T = (uint64_t)s.arg[l] * E;
        } else {
            if (E <= 2ull * s.arg[l])
                return false;
            T = 3 * (E - 2ull * s.arg[l]);
        }
        if (T > (1u << 20))
            return false;
        sz[l] = (uint32_t)T;
    }
    return true;
}

static gf2x_status check_spec_shape(const gf2x_plan_spec &s)
{
    if (s.nlev > (uint32_t)kMaxLevels)
        return GF2X_EINVAL;
    for (uint32_t l = 0; l < s.nlev; ++l) {
        if (s.kind[l] == GF2X_LEVEL_KARATSUBA) {
            if (s.arg[l] != 2 && s.arg[l] != 3 && s.arg[l] != 5)
                return GF2X_EINVAL;
        } else if (s.kind[l] == GF2X_LEVEL_TOOM3) {
            if (s.arg[l] < 1 || s.arg[l] > 64)
                return GF2X_EINVAL;
        } else {
            return GF2X_EINVAL;
        }
    }
    if (s.seq_top > 1)
        return GF2X_EINVAL;
    if (s.seq_top && s.nlev < 2)
        return GF2X_EINVAL;
    if (s.leaf_words && !leaf_supported(s.leaf_words))
        return GF2X_EINVAL;
    if (s.threads && (s.threads % 32 || s.threads > 1024))
        return GF2X_EINVAL;
    if (s.fuse_leaf > 1 || s.split_top > 1)
        return GF2X_EINVAL;
    if (s.split_top && s.nlev < 2)
        return GF2X_EINVAL;
    if (s.fuse_leaf) {
        if (s.nlev < 1 || s.kind[s.nlev - 1] != GF2X_LEVEL_KARATSUBA || s.arg[s.nlev - 1] != 2)
            return GF2X_EINVAL;
        if (s.leaf_words > kMaxFusedLeaf)
            return GF2X_EINVAL;
    }
    return GF2X_OK;
}

static void fill_karatsuba_tables(GLevel &L)
{
    const uint32_t k = L.k;
    if (k < 2 || k > 5)   // validated by check_spec_shape; bounds the tables below
        return;
    uint32_t j = 0;
    for (uint32_t i = 0; i < k && j < 16; ++i, ++j) {
        L.sel[j][0] = (uint8_t)i;
        L.sel[j][1] = 255;
    }
    uint32_t pairidx[5][5];
    for (uint32_t i = 0; i < k; ++i)
        for (uint32_t i2 = i + 1; i2 < k && j < 16; ++i2, ++j) {
            L.sel[j][0] = (uint8_t)i;
            L.sel[j][1] = (uint8_t)i2;
            pairidx[i][i2] = j;
        }
    for (uint32_t p = 0; p + 1 < 2 * k; ++p) {
        uint32_t c = 0;
        for (uint32_t i = 0; i < k; ++i)
            if (p >= i && p - i < k && c < (uint32_t)kMaxTerms)
                L.terms[p][c++] = (uint8_t)i;
        for (uint32_t i = 0; i < k; ++i) {
            uint32_t i2 = p - i;
            if (p >= i && i < i2 && i2 < k && c < (uint32_t)kMaxTerms)
                L.terms[p][c++] = (uint8_t)pairidx[i][i2];
        }
        L.nterms[p] = (uint8_t)c;
    }
}

// Modelled 32-bit integer operations (XOR/AND/shift) of one product.
static void op_model(const GPlan &P, const uint32_t *sz, const uint32_t *npar_all,
                     uint64_t *ops_total, uint64_t *ops_leaf)
{
    uint64_t ops = 0;
    for (uint32_t l = 0; l < P.nlev; ++l) {
        const GLevel &L = P.lev[l];
        uint64_t np_ = npar_all[l];
        if (L.kind == kKaratsuba) {
            uint64_t pairs = (uint64_t)L.k * (L.k - 1) / 2;
            uint64_t eval = pairs * 2ull * L.E;                       // operand sums
            uint64_t terms = 0;
            for (uint32_t p = 0; p + 1 < 2 * L.k; ++p)
                terms += L.nterms[p];
            uint64_t interp = terms * 2ull * L.E - 2ull * L.T;         // XORs of the reconstruction
            ops += np_ * (eval + interp);
        } else {
            uint64_t n1 = L.np, E = L.E;
            uint64_t eval = 2 * (2 * n1 + 4 * E);                     // v1, vx, vx1 for a and b
            uint64_t interp = 36 * n1;                                // two /x, two /(x+1) scans, recomposition
            ops += np_ * (eval + interp);
        }
    }
    const uint64_t S = P.S;
    // comb: 8 steps of (2S accumulator shifts, 4S masks, S b shifts, S(4S+3)
    // AND-XORs against a, aX^8, aX^16, aX^24) plus 3(S+1) shifts for those copies
    const uint64_t leaf = 32 * S * S + 83 * S + 3;
    const uint64_t nleaf_total = npar_all[P.nlev];
    *ops_leaf = nleaf_total * leaf;
    *ops_total = ops + *ops_leaf + 2ull * P.L64 * 2;                   // + fold / store
    (void)sz;
}

static gf2x_status build_split_plan(uint32_t n, const gf2x_plan_spec &s, GPlan *out, gf2x_plan_info *info,
                                    GPlan *child_out);

gf2x_status build_plan(uint32_t n, const gf2x_plan_spec *spec_in, GPlan *out, gf2x_plan_info *info,
                       GPlan *child_out)
{
    if (!spec_in)
        return GF2X_EINVAL;
    if (n < 1 || n > GF2X_MAX_N)
        return GF2X_EUNSUPPORTED;
    gf2x_plan_spec s = *spec_in;
    gf2x_status st = check_spec_shape(s);
    if (st != GF2X_OK)
        return st;

    if (s.split_top)
        return build_split_plan(n, s, out, info, child_out);

    const uint32_t L32 = (n + 31) / 32;
    uint32_t sz[kMaxLevels + 1];
    uint32_t S = s.leaf_words;
    if (S == 0) {
        for (uint32_t cand : kLeafSizes) {
            if (s.fuse_leaf && cand > kMaxFusedLeaf)
                continue;
            if (level_sizes(s, cand, sz) && sz[0] >= L32) {
                S = cand;
                break;
            }
        }
        if (S == 0)
            return GF2X_EUNSUPPORTED;
    }
    if (!level_sizes(s, S, sz))
        return GF2X_EINVAL;
    if (sz[0] < L32)
        return GF2X_EUNSUPPORTED;

    GPlan P;
    memset(&P, 0, sizeof(P));
    P.n = n;
    P.L32 = L32;
    P.L64 = (n + 63) / 64;
    P.Lfull64 = (uint32_t)((2ull * n - 1 + 63) / 64);
    P.T0 = sz[0];
    P.nlev = s.nlev;
    P.S = S;
    P.seq_top = s.seq_top;
    P.fuse_k2 = s.fuse_leaf;
    // depth of the deepest data held in shared memory (the fused level stays in registers)
    const uint32_t deepest = s.nlev - s.fuse_leaf;

    // parents per level over the whole tree, and per pass
    uint32_t npar_all[kMaxLevels + 1];
    npar_all[0] = 1;
    for (uint32_t l = 0; l < s.nlev; ++l) {
        uint32_t k = s.arg[l];
        uint32_t nch = s.kind[l] == GF2X_LEVEL_KARATSUBA ? k * (k + 1) / 2 : 5;
        uint64_t next = (uint64_t)npar_all[l] * nch;
        if (next > 100000)
            return GF2X_EUNSUPPORTED;
        npar_all[l + 1] = (uint32_t)next;
    }
    uint32_t npar_pass[kMaxLevels + 1];
    npar_pass[0] = 1;
    for (uint32_t l = 0; l < s.nlev; ++l) {
        uint32_t nch = s.kind[l] == GF2X_LEVEL_KARATSUBA ? s.arg[l] * (s.arg[l] + 1) / 2 : 5;
        npar_pass[l + 1] = (s.seq_top && l == 0) ? 1 : npar_pass[l] * nch;
    }
    P.nleaf_pass = npar_pass[deepest];

    // threads: enough for the leaf pass in as few balanced rounds as the leaf allows
    uint32_t maxT = max_threads_for_leaf(S);
    if (s.threads) {
        if (s.threads > maxT)
            return GF2X_EINVAL;
        P.threads = s.threads;
    } else {
        uint32_t rounds = (P.nleaf_pass + maxT - 1) / maxT;
        uint32_t t = round_up((P.nleaf_pass + rounds - 1) / rounds, 32);
        P.threads = std::max(128u, std::min(t, maxT));
    }

    for (uint32_t l = 0; l < s.nlev; ++l) {
        GLevel &L = P.lev[l];
        L.kind = s.kind[l] == GF2X_LEVEL_KARATSUBA ? kKaratsuba : kToom3;
        L.T = sz[l];
        L.E = sz[l + 1];
        if (L.kind == kKaratsuba) {
            L.k = s.arg[l];
            L.W = 0;
            L.np = L.E;
            L.nch = L.k * (L.k + 1) / 2;
            fill_karatsuba_tables(L);
        } else {
            L.k = 3;
            L.W = s.arg[l];
            L.np = L.E - 2 * L.W;
            L.nch = 5;
        }
        L.npar = npar_pass[l];
        L.div2E = make_div(2 * L.E);
        L.divnch = make_div(L.nch);
        L.divE = make_div(L.E);
        L.div2T = make_div(2 * L.T);
        L.divhE = make_div(std::max(1u, L.E / 2));
    }

    // ---- fused pairs of 2-way levels: levels l, l+1 (both K2, both shared-
    // memory passes, not the per-child top of seq_top) run as one pass from
    // depth l to depth l+2; depth l+1 is never stored.  Paired from the leaf
    // side upwards.
    const uint32_t ne = s.nlev - s.fuse_leaf;   // levels run as shared-memory passes
    bool mat[kMaxLevels + 1];
    for (uint32_t d = 0; d <= s.nlev; ++d)
        mat[d] = true;
    for (int l = (int)ne - 2; l >= (s.seq_top ? 1 : 0); --l) {
        GLevel &A = P.lev[l], &B = P.lev[l + 1];
        if (A.pair || B.pair || A.kind != kKaratsuba || B.kind != kKaratsuba || A.k != 2 || B.k != 2 || (B.E & 1u))
            continue;
        A.pair = 1;
        B.pair = 2;
        mat[l + 1] = false;
        --l;   // the level above this pair may pair with the one above it
    }

    // ---- shared-memory layout (words, 16-byte aligned regions)
    // data at depth d: npar_pass[d] slots of 2*sz[d] words; stored depths
    // alternate between two regions
    uint32_t D[kMaxLevels + 1];
    for (uint32_t d = 0; d <= s.nlev; ++d)
        D[d] = (d <= deepest && mat[d]) ? round_up(npar_pass[d] * 2 * sz[d], 4) : 0;
    uint32_t par_of[kMaxLevels + 1];   // region parity of every stored depth
    {
        uint32_t k = 0;
        for (uint32_t d = 0; d <= s.nlev; ++d)
            par_of[d] = mat[d] ? (k++ & 1u) : 0u;
    }
    // the depth a level's pass writes: l+1, or l+2 for the first of a pair
    auto out_depth = [&](uint32_t l) { return P.lev[l].pair == 1 ? l + 2 : l + 1; };
    uint32_t off = 0;
    uint32_t regA = 0, regB = 0, regP = 0;
    if (!s.seq_top) {
        for (uint32_t d = 0; d <= s.nlev; ++d)
            (par_of[d] == 0 ? regA : regB) = std::max(par_of[d] == 0 ? regA : regB, D[d]);
        uint32_t offA = off;
        off += regA;
        uint32_t offB = off;
        off += regB;
        P.top_off = offA;
        for (uint32_t l = 0; l < s.nlev; ++l) {
            const uint32_t din = P.lev[l].pair == 2 ? l - 1 : l;
            const uint32_t dout = P.lev[l].pair == 2 ? l + 1 : out_depth(l);
            P.lev[l].in_off = par_of[din] == 0 ? offA : offB;
            P.lev[l].ch_off = par_of[dout] == 0 ? offA : offB;
        }
    } else {
        // top slot, children products, then two regions Y / Z alternating over
        // the stored depths >= 1 (depth 1 in Y)
        uint32_t offX = off;
        off += D[0];
        regP = round_up(P.lev[0].nch * 2 * sz[1], 4);
        P.prod_off = off;
        off += regP;
        uint32_t regY = 0, regZ = 0;
        for (uint32_t d = 1; d <= s.nlev; ++d)
            (par_of[d] == par_of[1] ? regY : regZ) = std::max(par_of[d] == par_of[1] ? regY : regZ, D[d]);
        uint32_t offY = off;
        off += regY;
        uint32_t offZ = off;
        off += regZ;
        auto region = [&](uint32_t d) { return par_of[d] == par_of[1] ? offY : offZ; };
        P.top_off = offX;
        P.lev[0].in_off = offX;
        P.lev[0].ch_off = offY;
        for (uint32_t l = 1; l < s.nlev; ++l) {
            const uint32_t din = P.lev[l].pair == 2 ? l - 1 : l;
            const uint32_t dout = P.lev[l].pair == 2 ? l + 1 : out_depth(l);
            P.lev[l].in_off = region(din);
            P.lev[l].ch_off = region(dout);
        }
    }
    // Toom-3 temporaries: two arrays of 2E words per parent (c3 and the c2 numerator)
    uint32_t tmp = 0, part = P.threads;
    for (uint32_t l = 0; l < s.nlev; ++l) {
        const GLevel &L = P.lev[l];
        if (L.kind == kToom3) {
            tmp = std::max(tmp, round_up(L.npar * 4 * L.E, 4));
            part = std::max(part, L.npar * L.W);
        }
    }
    P.tmp_off = off;
    off += tmp;
    P.part_off = off;
    P.part_words = round_up(part, 4);
    off += P.part_words;
    P.smem_words = off;
    const uint64_t smem_bytes = 4ull * off;

    // index-range checks for the fast divisions: every x divided by d obeys x * d < 2^32
    for (uint32_t l = 0; l < s.nlev; ++l) {
        const GLevel &L = P.lev[l];
        const uint64_t xe = (uint64_t)npar_pass[l + 1] * 2 * L.E;   // eval: idx / 2E, child / nch
        const uint64_t xi = (uint64_t)npar_pass[l] * 2 * L.T;       // interp: idx / 2T, q / E
        if (xe * (2ull * L.E) >= (1ull << 32) || xi * (2ull * L.T) >= (1ull << 32) ||
            (2ull * L.T) * L.E >= (1ull << 32) || (uint64_t)npar_pass[l + 1] * L.nch >= (1ull << 32))
            return GF2X_EUNSUPPORTED;
    }
    if (smem_bytes > kMaxDynamicSmemBytes)
        return GF2X_EUNSUPPORTED;

    if (out)
        *out = P;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->n = n;
        info->top_words = P.T0;
        info->leaf_words = S;
        info->nleaves = npar_all[s.nlev];
        info->threads = P.threads;
        info->smem_bytes = (uint32_t)smem_bytes;
        for (uint32_t d = 0; d <= s.nlev; ++d)
            info->level_words[d] = sz[d];
        op_model(P, sz, npar_all, &info->ops_full, &info->ops_leaf);
        info->clmul64 = (S % 2 == 0) ? (uint64_t)npar_all[s.nlev] * (S / 2) * (S / 2) : 0;
        info->bytes_in = 2ull * 8 * P.L64;
        info->bytes_out_full = 8ull * P.Lfull64;
        info->bytes_out_reduced = 8ull * P.L64;
        info->scratch_bytes = 0;
    }
    return GF2X_OK;
}

// Split plan: level 0 across CTAs.  The children are products of E0 words
// (n_child = 32 E0 bits, full products of 2 E0 words written over their
// operand slot in scratch); the top plan holds level 0 alone with its own
// shared-memory layout (operands / product, children, Toom temporaries).
static gf2x_status build_split_plan(uint32_t n, const gf2x_plan_spec &s, GPlan *out, gf2x_plan_info *info,
                                    GPlan *child_out)
{
    if (out && !child_out)
        return GF2X_EINVAL;
    gf2x_plan_spec cs;
    memset(&cs, 0, sizeof(cs));
    cs.nlev = s.nlev - 1;
    for (uint32_t l = 1; l < s.nlev; ++l) {
        cs.kind[l - 1] = s.kind[l];
        cs.arg[l - 1] = s.arg[l];
    }
    cs.leaf_words = s.leaf_words;
    cs.threads = s.threads;
    cs.seq_top = s.seq_top;
    cs.fuse_leaf = s.fuse_leaf;
    if (cs.seq_top && cs.nlev < 2)
        return GF2X_EINVAL;
    // the child size: smallest leaf such that the full tree covers n
    const uint32_t L32 = (n + 31) / 32;
    uint32_t sz[kMaxLevels + 1];
    uint32_t S = s.leaf_words;
    gf2x_plan_spec probe = s;
    probe.split_top = 0;
    if (S == 0) {
        for (uint32_t cand : kLeafSizes) {
            if (s.fuse_leaf && cand > kMaxFusedLeaf)
                continue;
            if (level_sizes(probe, cand, sz) && sz[0] >= L32) {
                S = cand;
                break;
            }
        }
        if (S == 0)
            return GF2X_EUNSUPPORTED;
    }
    if (!level_sizes(probe, S, sz))
        return GF2X_EINVAL;
    if (sz[0] < L32)
        return GF2X_EUNSUPPORTED;
    const uint32_t T0 = sz[0], E0 = sz[1];
    if (E0 & 1u)
        return GF2X_EINVAL;
    cs.leaf_words = S;
    if (32ull * E0 > GF2X_MAX_N)
        return GF2X_EUNSUPPORTED;
    GPlan C;
    gf2x_plan_info ci;
    gf2x_status st = build_plan(32u * E0, &cs, &C, &ci);
    if (st != GF2X_OK)
        return st;

    GPlan P;
    memset(&P, 0, sizeof(P));
    P.n = n;
    P.L32 = L32;
    P.L64 = (n + 63) / 64;
    P.Lfull64 = (uint32_t)((2ull * n - 1 + 63) / 64);
    P.T0 = T0;
    P.nlev = 1;
    P.S = C.S;
    P.split = 1;
    P.threads = 256;
    GLevel &L = P.lev[0];
    L.kind = s.kind[0] == GF2X_LEVEL_KARATSUBA ? kKaratsuba : kToom3;
    L.T = T0;
    L.E = E0;
    if (L.kind == kKaratsuba) {
        L.k = s.arg[0];
        L.W = 0;
        L.np = E0;
        L.nch = L.k * (L.k + 1) / 2;
        fill_karatsuba_tables(L);
    } else {
        L.k = 3;
        L.W = s.arg[0];
        L.np = E0 - 2 * L.W;
        L.nch = 5;
    }
    L.npar = 1;
    L.div2E = make_div(2 * E0);
    L.divnch = make_div(L.nch);
    L.divE = make_div(E0);
    L.div2T = make_div(2 * T0);
    L.divhE = make_div(std::max(1u, E0 / 2));
    uint32_t off = 0;
    P.top_off = off;
    L.in_off = off;
    off += round_up(2 * T0, 4);
    L.ch_off = off;
    off += round_up(L.nch * 2 * E0, 4);
    P.tmp_off = off;
    if (L.kind == kToom3)
        off += round_up(4 * E0, 4);
    P.part_off = off;
    P.part_words = round_up(std::max(P.threads, L.W), 4);
    off += P.part_words;
    P.smem_words = off;
    if (4ull * off > kMaxDynamicSmemBytes)
        return GF2X_EUNSUPPORTED;
    const uint64_t xe = (uint64_t)L.nch * 2 * E0, xi = 2ull * T0;
    if (xe * (2ull * E0) >= (1ull << 32) || xi * xi >= (1ull << 32) || xi * E0 >= (1ull << 32))
        return GF2X_EUNSUPPORTED;

    if (out) {
        *out = P;
        *child_out = C;
    }
    if (info) {
        memset(info, 0, sizeof(*info));
        info->n = n;
        info->top_words = T0;
        info->leaf_words = C.S;
        info->nleaves = L.nch * ci.nleaves;
        info->threads = C.threads;
        info->smem_bytes = (uint32_t)std::max<uint64_t>(4ull * off, ci.smem_bytes);
        info->level_words[0] = T0;
        for (uint32_t d = 0; d < cs.nlev + 1 && d + 1 <= (uint32_t)kMaxLevels; ++d)
            info->level_words[d + 1] = ci.level_words[d];
        // top level work (same model as an in-CTA level) plus the children's
        uint64_t top = 0;
        if (L.kind == kKaratsuba) {
            uint64_t pairs = (uint64_t)L.k * (L.k - 1) / 2, terms = 0;
            for (uint32_t q = 0; q + 1 < 2 * L.k; ++q)
                terms += L.nterms[q];
            top = pairs * 2ull * E0 + terms * 2ull * E0 - 2ull * T0;
        } else {
            top = 2ull * (2ull * L.np + 4ull * E0) + 36ull * L.np;
        }
        info->ops_leaf = (uint64_t)L.nch * ci.ops_leaf;
        info->ops_full = top + (uint64_t)L.nch * (ci.ops_full - 4ull * (32u * E0 / 64)) + 4ull * P.L64;
        info->clmul64 = (uint64_t)L.nch * ci.clmul64;
        info->bytes_in = 2ull * 8 * P.L64;
        info->bytes_out_full = 8ull * P.Lfull64;
        info->bytes_out_reduced = 8ull * P.L64;
        info->scratch_bytes = 4ull * L.nch * 2 * E0;
    }
    return GF2X_OK;
}

// ---- default plan: minimise the modelled operation count over a family of
// plans (optional Toom-3 top, non-increasing Karatsuba splits, every compiled
// leaf) among those that leave room for two CTAs per SM; fall back to one
// CTA per SM, then to the sequential top level.
static void enumerate_kseq(std::vector<std::vector<uint32_t>> &out, std::vector<uint32_t> &cur, uint32_t maxk,
                           uint32_t depth)
{
    out.push_back(cur);
    if (depth == 0)
        return;
    for (uint32_t k : {5u, 3u, 2u}) {
        if (k > maxk)
            continue;
        cur.push_back(k);
        enumerate_kseq(out, cur, k, depth - 1);
        cur.pop_back();
    }
}

gf2x_status default_spec(uint32_t n, gf2x_plan_spec *out)
{
    if (!out)
        return GF2X_EINVAL;
    if (n < 1 || n > GF2X_MAX_N)
        return GF2X_EUNSUPPORTED;
    std::vector<std::vector<uint32_t>> kseqs;
    std::vector<uint32_t> cur;
    enumerate_kseq(kseqs, cur, 5, 6);
    const uint32_t toomW[] = {0, 1, 2, 4, 8, 16};
    const uint64_t budgets[] = {kMaxDynamicSmemBytes / 2 - 2048, kMaxDynamicSmemBytes};
    for (uint64_t budget : budgets) {
        for (uint32_t seq = 0; seq <= 1; ++seq) {
            bool found = false;
            uint64_t best_ops = ~0ull;
            gf2x_plan_spec best;
            for (uint32_t W : toomW) {
                for (const auto &ks : kseqs) {
                    gf2x_plan_spec s;
                    memset(&s, 0, sizeof(s));
                    uint32_t l = 0;
                    if (W) {
                        s.kind[l] = GF2X_LEVEL_TOOM3;
                        s.arg[l++] = W;
                    }
                    for (uint32_t k : ks) {
                        if (l >= (uint32_t)kMaxLevels)
                            break;
                        s.kind[l] = GF2X_LEVEL_KARATSUBA;
                        s.arg[l++] = k;
                    }
                    s.nlev = l;
                    s.seq_top = seq;
                    if (seq && l < 2)
                        continue;
                    for (uint32_t S : kLeafSizes) {
                        s.leaf_words = S;
                        s.fuse_leaf = (l >= 1 && s.kind[l - 1] == GF2X_LEVEL_KARATSUBA && s.arg[l - 1] == 2 &&
                                       S <= kMaxFusedLeaf) ? 1u : 0u;
                        gf2x_plan_info info;
                        if (build_plan(n, &s, nullptr, &info) != GF2X_OK)
                            continue;
                        if (info.smem_bytes > budget)
                            continue;
                        // prefer fewer ops; tie-break on smaller smem
                        uint64_t score = info.ops_full;
                        if (score < best_ops) {
                            best_ops = score;
                            best = s;
                            found = true;
                        }
                    }
                }
            }
            if (found) {
                *out = best;
                return GF2X_OK;
            }
        }
    }
    // no plan fits one CTA: split the top level across CTAs
    {
        bool found = false;
        uint64_t best_ops = ~0ull;
        gf2x_plan_spec best;
        for (uint32_t W : toomW) {
            for (const auto &ks : kseqs) {
                gf2x_plan_spec sp;
                memset(&sp, 0, sizeof(sp));
                uint32_t l = 0;
                if (W) {
                    sp.kind[l] = GF2X_LEVEL_TOOM3;
                    sp.arg[l++] = W;
                }
                for (uint32_t k : ks) {
                    if (l >= (uint32_t)kMaxLevels)
                        break;
                    sp.kind[l] = GF2X_LEVEL_KARATSUBA;
                    sp.arg[l++] = k;
                }
                sp.nlev = l;
                sp.split_top = 1;
                if (l < 2)
                    continue;
                for (uint32_t seq = 0; seq <= 1; ++seq) {
                    sp.seq_top = seq;
                    if (seq && l < 3)
                        continue;
                    for (uint32_t S : kLeafSizes) {
                        sp.leaf_words = S;
                        sp.fuse_leaf = (sp.kind[l - 1] == GF2X_LEVEL_KARATSUBA && sp.arg[l - 1] == 2 &&
                                        S <= kMaxFusedLeaf) ? 1u : 0u;
                        gf2x_plan_info info;
                        if (build_plan(n, &sp, nullptr, &info) != GF2X_OK)
                            continue;
                        if (info.ops_full < best_ops) {
                            best_ops = info.ops_full;
                            best = sp;
                            found = true;
                        }
                    }
                }
            }
        }
        if (found) {
            *out = best;
            return GF2X_OK;
        }
    }
    return GF2X_EUNSUPPORTED;
}

gf2x_status default_split_spec(uint32_t n, gf2x_plan_spec *out)
{
    if (!out)
        return GF2X_EINVAL;
    if (n < 1 || n > GF2X_MAX_N)
        return GF2X_EUNSUPPORTED;
    std::vector<std::vector<uint32_t>> kseqs;
    std::vector<uint32_t> cur;
    enumerate_kseq(kseqs, cur, 5, 6);
    const uint32_t toomW[] = {0, 1, 2, 4, 8, 16};
    bool found = false;
    uint64_t best_ops = ~0ull;
    gf2x_plan_spec best;
    for (uint32_t W : toomW) {
        for (const auto &ks : kseqs) {
            gf2x_plan_spec sp;
            memset(&sp, 0, sizeof(sp));
            uint32_t l = 0;
            if (W) {
                sp.kind[l] = GF2X_LEVEL_TOOM3;
                sp.arg[l++] = W;
            }
            for (uint32_t k : ks) {
                if (l >= (uint32_t)kMaxLevels)
                    break;
                sp.kind[l] = GF2X_LEVEL_KARATSUBA;
                sp.arg[l++] = k;
            }
            sp.nlev = l;
            sp.split_top = 1;
            if (l < 2)
                continue;
            for (uint32_t S : kLeafSizes) {
                sp.leaf_words = S;
                sp.fuse_leaf = (sp.kind[l - 1] == GF2X_LEVEL_KARATSUBA && sp.arg[l - 1] == 2 && S <= kMaxFusedLeaf)
                                   ? 1u : 0u;
                gf2x_plan_info info;
                if (build_plan(n, &sp, nullptr, &info) != GF2X_OK)
                    continue;
                if (info.ops_full < best_ops) {
                    best_ops = info.ops_full;
                    best = sp;
                    found = true;
                }
            }
        }
    }
    if (!found)
        return GF2X_EUNSUPPORTED;
    *out = best;
    return GF2X_OK;
}

gf2x_status parse_spec(const char *text, gf2x_plan_spec *out)
{
    if (!text || !out)
        return GF2X_EINVAL;
    gf2x_plan_spec s;
    memset(&s, 0, sizeof(s));
    std::string t(text);
    std::vector<std::string> fields;
    size_t pos = 0;
    while (true) {
        size_t q = t.find('/', pos);
        fields.push_back(t.substr(pos, q == std::string::npos ? std::string::npos : q - pos));
        if (q == std::string::npos)
            break;
        pos = q + 1;
    }
    if (fields.size() > 6)
        return GF2X_EINVAL;
    // levels
    const std::string &lv = fields[0];
    size_t i = 0;
    while (i < lv.size()) {
        size_t j = lv.find('.', i);
        std::string tok = lv.substr(i, j == std::string::npos ? std::string::npos : j - i);
        if (!tok.empty()) {
            if (s.nlev >= (uint32_t)kMaxLevels || tok.size() < 2)
                return GF2X_EINVAL;
            char kind = tok[0];
            char *end = nullptr;
            unsigned long v = strtoul(tok.c_str() + 1, &end, 10);
            if (*end != '\0')
                return GF2X_EINVAL;
            if (kind == 'K')
                s.kind[s.nlev] = GF2X_LEVEL_KARATSUBA;
            else if (kind == 'T')
                s.kind[s.nlev] = GF2X_LEVEL_TOOM3;
            else
                return GF2X_EINVAL;
            s.arg[s.nlev++] = (uint32_t)v;
        }
        if (j == std::string::npos)
            break;
        i = j + 1;
    }
    uint32_t *dst[5] = {&s.leaf_words, &s.threads, &s.seq_top, &s.fuse_leaf, &s.split_top};
    for (size_t f = 1; f < fields.size(); ++f) {
        if (fields[f].empty())
            continue;
        char *end = nullptr;
        unsigned long v = strtoul(fields[f].c_str(), &end, 10);
        if (*end != '\0')
            return GF2X_EINVAL;
        *dst[f - 1] = (uint32_t)v;
    }
    gf2x_status st = check_spec_shape(s);
    if (st != GF2X_OK)
        return st;
    *out = s;
    return GF2X_OK;
}

}  // namespace gf2x
