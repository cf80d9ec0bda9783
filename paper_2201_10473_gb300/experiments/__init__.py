"""Measurement programs behind the design choices (not part of the product path).

  alu_pipes    LOP3 / SHF / IMAD throughput per SM (the integer roofline peak)
  fma_pipes    IMAD.HI and IMAD.WIDE throughput (why the leaf stays on the ALU pipe)
  mma_pipes    mma.sync s8 / f16 / e4m3 throughput
  tc_toeplitz  fp8 tensor-core Toeplitz multiplier vs the comb leaf (bit-exact check + timing)

Run one on a GPU:  python -m paper_2201_10473_gb300.experiments.run <name>
"""
