"""GB300-native reverse-mode AD of reduce, scan and reduce-by-index.

The compute path is ``libadcomb.so`` (hand-written CUDA for sm_103a behind a
C-ABI, see ``include/adcomb.h``); :mod:`.adcomb` is its thin ctypes binding and
:mod:`.autograd` wraps it in ``torch.autograd.Function``s.  Importing this
package does not load the library; the first call that needs it does, and it
raises if the library is missing -- there is no CPU fallback.
"""
__all__ = ["adcomb", "autograd", "synth"]
