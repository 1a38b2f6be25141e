"""GB300-native TRPL+K eigensolver hot path.

Importing the package loads nothing native; ``paper_1711_10128_gb300.binding``
loads ``libtrplk.so`` on first use and fails loudly if it is missing.
"""
