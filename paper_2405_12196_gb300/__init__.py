"""GB300 (sm_103a) library for contracting abelian-symmetric block-sparse tensors.

The C ABI is ``include/ytn.h``; ``paper_2405_12196_gb300.ytn`` is its Python binding.
Import the binding explicitly (``from paper_2405_12196_gb300 import ytn``): it loads
``libytn.so`` and raises if the library has not been built.
"""
