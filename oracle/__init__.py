"""FP64 CPU oracle of the VRSplat rasterizer hot path (arXiv 2505.10144).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import it.  It shares no code
with the CUDA path: ``native`` wraps the plain C definition of the forward pass
(``vrs_oracle.c``); ``grad`` restates the same per-pair arithmetic in float64 PyTorch so
that autograd gives the gradient oracle; ``loss`` and ``net`` hold the SSIM loss and the
periphery network as plain definitions.
"""
