"""GNN-corrected IC(0)-preconditioned CG on GB300 (arxiv 2412.07127).

The compute path lives in the CUDA library built from csrc/ and is reached
through the C-ABI binding in `gicpcg`. `inputs` holds the seeded synthetic
workload generators. Importing the package does not load the CUDA library;
the first call into `gicpcg` does, and fails loudly if it is missing.
"""
