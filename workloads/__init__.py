"""Seeded input generators shared by the library's callers and the oracle.

Holds surface charts sampled at a node rule, right-hand sides and named
workloads.  Contains none of the layer-potential arithmetic.
"""
