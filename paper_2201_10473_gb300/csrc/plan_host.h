// plan_host.h -- host-side plan building (see plan_host.cpp).
#pragma once
#include "gf2x_gb300.h"
#include "plan.h"

namespace gf2x {

constexpr int kNumLeafSizes = 6;
constexpr uint32_t kMaxFusedLeaf = 10;  // largest leaf whose fused 2-way Karatsuba fits the registers
extern const uint32_t kLeafSizes[kNumLeafSizes];

// Dynamic shared memory one CTA may use: the 227 KB opt-in maximum of the
// SM minus the statically declared plan copy.
constexpr uint64_t kMaxDynamicSmemBytes = 232448ull - sizeof(GPlan) - 256;

uint32_t max_threads_for_leaf(uint32_t S);
bool leaf_supported(uint32_t S);
// For a split plan (spec->split_top) `out` receives the top-level plan and
// `child_out` the plan of the children (which must then be non-null).
gf2x_status build_plan(uint32_t n, const gf2x_plan_spec *spec, GPlan *out, gf2x_plan_info *info,
                       GPlan *child_out = nullptr);
gf2x_status default_spec(uint32_t n, gf2x_plan_spec *out);
gf2x_status parse_spec(const char *text, gf2x_plan_spec *out);
// The split plan (split_top = 1) with the fewest modelled operations for n.
gf2x_status default_split_spec(uint32_t n, gf2x_plan_spec *out);

}  // namespace gf2x
