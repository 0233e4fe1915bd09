"""GB300 spherical-harmonic transforms on the nestable Clenshaw-Curtis grid.

Hand-written sm_103a CUDA kernels behind a C ABI (``include/sht.h``); this
package is the thin Python binding.  ``Plan`` is imported lazily so that the
input generators in ``workloads`` stay usable without the built library.
"""


def __getattr__(name):
    if name in ("Plan", "Group", "Analysis", "Synthesis", "analysis", "synthesis",
                "SHTError"):
        from . import sht
        return getattr(sht, name)
    raise AttributeError(name)
