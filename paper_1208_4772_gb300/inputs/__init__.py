"""Seeded synthetic inputs: meshes, wall curving (host setup) and states.

Shared by the tests, the benchmark and the serving loop; holds no part of
the discretisation's arithmetic.
"""
