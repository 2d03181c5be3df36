"""GB300-native passing-point search (SBIP-DPPS, ZJUNlict 2019, Sec. 4.2-4.3).

The search runs in hand-written sm_103a CUDA kernels behind the C-ABI
library ``libpps.so`` (declared in ``include/pps.h``).  ``pps`` is its thin
ctypes binding; ``synth`` draws seeded synthetic states.  Importing the
package loads nothing: the CUDA library is opened on first use and a missing
or unbuilt library raises instead of falling back to anything else.
"""
__all__ = ["pps", "synth"]
