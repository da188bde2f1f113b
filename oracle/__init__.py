"""FP64 CPU oracle for Lazy SPCA and SPCA (Wojnowicz et al., arXiv 1709.07175).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of what the GPU library computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference arm of ``bench.py``
may import it.  The CUDA library never calls it, shares no code with it, and
fails loudly when its own extension is missing.

Modules
-------
philox   Philox4x32-10 (Salmon et al., SC'11) and the two random test matrices
         of Sec. I-A (Gaussian and very sparse Omega).
lspca    The method: Eq. 1 sketch, Algorithms 1-4, the eigen route of the
         table footnote, the reduction maps of Sec. III-B.2, Prop. 1-3 helpers.
metrics  Subspace sine, chordal distance (Experiment 2), Procrustes alignment.

Every function cites the passage of the paper it follows.  Functions without
an independent pin say "parity unpinned" in their docstring (none at present).
"""
