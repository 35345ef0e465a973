"""GB300-native RKDG right-hand side and SSP-RK stage update for the 2D Euler
equations on curved triangles (after Siebenborn, Schulz & Schmidt, arXiv
1208.4772).

The computation lives in libdgcurved.so (CUDA for sm_103a, C ABI in
include/dgcurved.h); ``binding`` is its ctypes binding; ``inputs`` holds the
seeded synthetic meshes and states; ``serve`` the continuous-batching
request loop.
"""
