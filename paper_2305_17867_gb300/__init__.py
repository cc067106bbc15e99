"""GB300-native compressed-Taylor FMM (Fernando & Kloeckner, arXiv 2305.17867).

The product is the C-ABI CUDA library ``libctfmm`` (``include/ctfmm.h``);
``paper_2305_17867_gb300.fmm`` is its thin PyTorch-facing binding.
"""

__all__ = ["FMM", "fmm_potential"]


def __getattr__(name):
    if name in __all__:
        from . import fmm

        return getattr(fmm, name)
    raise AttributeError(name)
