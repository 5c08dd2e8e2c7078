"""GB300-native (sm_103a) tile rasterizer for 3D Gaussian Splatting with the
Speedy-Splat Gaussian-to-tile localization (3-sigma box, SnugBox, AccuTile).

Importing the package loads nothing; ``paper_2412_00578_gb300.raster`` binds
the CUDA library and raises if it has not been built.
"""
__version__ = "0.1.0"
