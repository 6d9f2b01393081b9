"""GB300-native multichannel FIR / IIR filter chains (TorchFX, arXiv 2504.08624).

The compute lives in ``libtfx.so`` (hand-written CUDA for sm_103a behind the C
ABI in ``include/tfx.h``); this package is its thin Python binding.  Importing
the package does not load the library; the first call does, and fails loudly
if it has not been built.
"""
__version__ = "0.1.0"


def __getattr__(name):
    if name in ("chain", "fir", "sos", "Plan", "TfxError", "chain_ad", "ChainFunction", "FilterChain", "mse",
                "mse_loss", "LearnableBiquadChain", "Batch", "design"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
