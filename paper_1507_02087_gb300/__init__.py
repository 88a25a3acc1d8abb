"""GB300-native SP2 density-matrix purification (arXiv:1507.02087).

The compute path lives in the C-ABI library built from `csrc/` (see
`paper_1507_02087_gb300.sp2` for the Python binding).  `inputs` holds the seeded
synthetic Fock-matrix generators.
"""
