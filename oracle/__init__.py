"""The oracle: a plain CPU definition of the rasterizer's results.

TEST INFRASTRUCTURE ONLY -- imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product package.
"""
