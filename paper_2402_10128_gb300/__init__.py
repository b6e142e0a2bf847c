"""GB300-native rasterizer for Generalized Exponential Splatting (GES).

The compute path is a C-ABI CUDA library (``libges``) built for sm_103a; this
package holds its Python binding (``ges``), a ``torch.autograd.Function``
wrapper and the seeded scene generators.  Importing the package loads nothing;
``paper_2402_10128_gb300.ges`` loads the library and raises if it is missing.
"""
__all__ = ["scenes"]
