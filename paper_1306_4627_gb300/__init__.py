"""GB300-native LCS (longest common subsequence) table fill and traceback.

The compute path is a CUDA library (`liblcs.so`, built from `csrc/`) behind a C ABI; `lcs` is its thin Python
binding. Import `paper_1306_4627_gb300.lcs` for the API; `paper_1306_4627_gb300.gen` holds the seeded input
generators. Importing the package itself loads nothing.
"""
