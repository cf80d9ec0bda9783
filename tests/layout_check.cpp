// Host-side check of every shared-memory pass of a plan: bounds and read/write
// disjointness of each evaluation, leaf and reconstruction pass, for plans read
// from stdin ("n spec" per line).  Built and run by tests/test_plan_layout.py.
#include <cstdio>
#include <cstring>
#include <string>
#include <iostream>
#include "gf2x_gb300.h"
#include "plan.h"
#include "plan_host.h"
using namespace gf2x;

static int bad = 0;
static void rng(const char *what, const GPlan &P, uint64_t lo, uint64_t len, const char *spec) {
    if (lo + len > P.smem_words) { printf("OOB %s [%llu,%llu) > %u  %s\n", what, (unsigned long long)lo, (unsigned long long)(lo+len), P.smem_words, spec); ++bad; }
}
static void disj(const char *what, uint64_t a, uint64_t al, uint64_t b, uint64_t bl, const char *spec) {
    if (a < b + bl && b < a + al) { printf("OVERLAP %s [%llu,%llu) [%llu,%llu) %s\n", what, (unsigned long long)a,(unsigned long long)(a+al),(unsigned long long)b,(unsigned long long)(b+bl), spec); ++bad; }
}

static void check(const GPlan &P, const char *spec) {
    const uint32_t ne = P.nlev - P.fuse_k2;
    rng("top", P, P.top_off, 2ull * P.T0, spec);
    uint32_t l0 = P.seq_top ? 1 : 0;
    if (P.seq_top && P.nlev > 0) {
        const GLevel &L = P.lev[0];
        rng("L0 child", P, L.ch_off, 2ull * L.E, spec);
        disj("L0 eval", L.in_off, 2ull * L.T, L.ch_off, 2ull * L.E, spec);
        rng("prod", P, P.prod_off, (uint64_t)L.nch * 2 * L.E, spec);
        disj("prod/child", P.prod_off, (uint64_t)L.nch * 2 * L.E, L.ch_off, 2ull * L.E, spec);
    }
    for (uint32_t l = l0; l < ne; ++l) {
        const GLevel &L = P.lev[l];
        if (L.pair == 2) continue;
        uint64_t inlen = (uint64_t)L.npar * 2 * L.T;
        uint64_t outlen = L.pair == 1 ? (uint64_t)L.npar * 18 * P.lev[l + 1].E : (uint64_t)L.npar * L.nch * 2 * L.E;
        if (L.pair == 1 && P.lev[l + 1].pair != 2) { printf("PAIR mismatch %s\n", spec); ++bad; }
        rng("in", P, L.in_off, inlen, spec);
        rng("out", P, L.ch_off, outlen, spec);
        disj("pass", L.in_off, inlen, L.ch_off, outlen, spec);
        if (P.seq_top && l >= 1) {
            disj("pass/prod", P.prod_off, (uint64_t)P.lev[0].nch * 2 * P.lev[0].E, L.ch_off, outlen, spec);
            disj("pass/top", P.top_off, 2ull * P.T0, L.ch_off, outlen, spec);
            disj("passin/prod", P.prod_off, (uint64_t)P.lev[0].nch * 2 * P.lev[0].E, L.in_off, inlen, spec);
        }
    }
    if (P.nlev > 0) {
        uint64_t base = P.fuse_k2 ? P.lev[P.nlev - 1].in_off : P.lev[P.nlev - 1].ch_off;
        uint64_t slot = P.fuse_k2 ? 4ull * P.S : 2ull * P.S;
        rng("leaf", P, base, P.nleaf_pass * slot, spec);
        if (P.seq_top) {
            disj("leaf/prod", P.prod_off, (uint64_t)P.lev[0].nch * 2 * P.lev[0].E, base, P.nleaf_pass * slot, spec);
            disj("leaf/top", P.top_off, 2ull * P.T0, base, P.nleaf_pass * slot, spec);
        }
        // the deepest pass's output must be where the leaves are
        if (!P.fuse_k2) {
            int l = ne - 1; while (l >= 0 && P.lev[l].pair == 2) --l;
            if (l >= (int)l0 && P.lev[l].ch_off != base) { printf("LEAFBASE %s\n", spec); ++bad; }
        }
    }
    rng("tmp", P, P.tmp_off, 0, spec);
    rng("part", P, P.part_off, P.part_words, spec);
}

int main() {
    std::string line;
    long count = 0, pairs = 0;
    while (std::getline(std::cin, line)) {
        char spec[256]; unsigned n;
        if (sscanf(line.c_str(), "%u %255s", &n, spec) != 2) continue;
        gf2x_plan_spec s;
        if (parse_spec(spec, &s) != GF2X_OK) continue;
        GPlan P, C; gf2x_plan_info info;
        if (build_plan(n, &s, &P, &info, &C) != GF2X_OK) continue;
        if (P.split) check(C, spec); else check(P, spec);
        for (int l = 0; l < 8; ++l) pairs += (P.split ? C : P).lev[l].pair == 1;
        ++count;
    }
    printf("checked %ld plans, %ld pairs, %d problems\n", count, pairs, bad);
    return bad ? 1 : 0;
}
