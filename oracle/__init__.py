"""CPU oracle of MaskGaussian's masked rasterisation (arXiv 2412.20522).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
anything under ``oracle/``: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg (and its ``--impl reference`` arm) may.

The oracle is a plain, slow, independent restatement of the method:

* ``fp32_path``   -- the discrete decisions (mask sample, near/det culls,
                     radius, tile rectangle, depth key) in a specified
                     sequence of correctly rounded FP32 operations, with the
                     project's own FP32 ``log``/``exp`` and Philox4x32-10.
* ``preprocess``  -- the per-Gaussian splat (Sec. 3.1) in FP64 with PyTorch
                     CPU ops; its backward is the exact derivative (autograd).
* ``binning``     -- instance emission, stable sort, tile ranges (Sec. 3.1).
* ``render.c``    -- masked compositing, Eq. 3-4, in FP64: tiled and
                     brute-force per-pixel forms, plain 3DGS Eq. 1-2, and the
                     mask/colour/alpha gradients of Eq. 6 and Appendix A.
* ``pipeline``    -- the forward+backward of one training step built from
                     the above, with the mask loss of Eq. 7-8 and the
                     ablations of Sec. 4.3 (threshold mask, mask x opacity).
* ``pruning``     -- the pruning rule of Sec. 3.5 (keep what is sampled
                     present in any of n draws) and the order-keeping
                     compaction of the survivors.

It shares no code with the CUDA path; the only common module is the seeded
input generator ``paper_2412_20522_gb300.scenes``.
"""
