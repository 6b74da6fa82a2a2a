"""GB300-native miniBUDE pose-energy engine (arxiv 2509.21039, Sec. 2.2, Listing 4).

The compute path is the C-ABI library ``libbude.so`` built from ``csrc/``;
``paper_2509_21039_gb300.bude`` is its thin ctypes binding.  ``synth`` draws
the seeded synthetic decks.  Submodules are imported lazily so that drawing
inputs does not load the CUDA library.
"""
__all__ = ["bude", "synth"]
