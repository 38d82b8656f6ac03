// ifctn_plan.h -- host-side launch planning of the streaming contraction.
#pragma once
#include <vector>

#include "ifctn_internal.cuh"

namespace ifctn {

// Dynamic shared memory a planned contraction kernel may use.
constexpr int SMEM_LIMIT = 220 * 1024;
// Tensors up to this size stay in L2 across a sweep: they run the persistent
// path by default, and their N = 3 modes A and B use one work unit per slab
// with mode 0 deferred to the reduction (more CTAs, smaller partials) instead
// of folding mode 0 in registers.
constexpr long long L2_RESIDENT_BYTES = 96LL << 20;

inline int cdiv(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

// SMs of the current device (queried once).
int num_sms();

// CTA kernels (persistent path, and the graph path's fallback).
ContractPlan plan_contract(const Shape& s, int k, int sz, std::vector<UnitDesc>& units);
// The launch-shape choices left open (rows per lane allowed unless
// IFCTN_CW_RPL=1; ring stages, task bytes and chunking by the cost model).
WarpKnobs default_warp_knobs();
// Warp-pipelined kernels (HBM-sized tensors); plan.warp = 0 when the shape
// does not suit them.
ContractPlan plan_contract_warp(const Shape& s, int k, int sz, std::vector<UnitDesc>& units, const WarpKnobs& kn);

}  // namespace ifctn
