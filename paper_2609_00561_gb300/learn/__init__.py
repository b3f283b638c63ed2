"""Learned blocking: features of a matrix -> ABMC block size and Leiden CPM
resolution, an MLP trained on the GPU by the library's own kernels."""
