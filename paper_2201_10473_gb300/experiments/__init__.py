"""Measurement programs behind the design choices (not part of the product path).

  tc_toeplitz     fp8 warp-MMA (mma.sync) Toeplitz multiplier vs the comb leaf (bit-exact check + timing)
  bitsliced_leaf  bitsliced leaves (32 per group) vs the comb leaf (bit-exact check + timing)

Run one on a GPU:  python -m paper_2201_10473_gb300.experiments.run <name>
"""
