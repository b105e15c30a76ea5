"""o3g: GB300-native point-to-plane ICP and hybrid-kNN normal estimation (Open3D, arXiv 1801.09847).

The compute path is the CUDA library ``libo3g.so`` behind the C ABI declared in
``include/o3g.h``; ``paper_1801_09847_gb300.o3g`` is its thin ctypes binding.
``paper_1801_09847_gb300.synth`` builds seeded synthetic inputs.  Importing the
package does not load the CUDA library; the binding does on first use and
raises if it is missing.
"""
__all__ = ["o3g", "synth"]
