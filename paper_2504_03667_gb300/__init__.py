"""GB300-native dense adjacency-matrix Dijkstra (Algorithm 1 of arXiv 2504.03667).

The CUDA library libdj.so (include/dj.h) does all the work; ``dj`` is its
Python binding with the same entry-point names.  Importing this package loads
nothing: ``from paper_2504_03667_gb300 import dj`` then ``dj.load_library()``
(or any call) loads the library and raises if it has not been built.
"""
__all__ = ["dj", "build"]
