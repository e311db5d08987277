"""GB300 (sm_103a) wavefront path guiding: SVO radiant-exitance cache, ray
binning, per-bin cone-traced radiance fields and their PDF/CDF sampling.

The CUDA library (libwfpg.so, C ABI in include/wfpg.h) is loaded by
``paper_2405_06997_gb300.wfpg``; the seeded synthetic inputs live in
``paper_2405_06997_gb300.inputs`` (numpy only, importable without a GPU).
"""
__all__ = ["inputs", "wfpg", "build"]
