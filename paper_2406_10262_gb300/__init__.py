"""GB300-native NSW fair ranking by gradient ascent over batched Sinkhorn solves.

The compute path lives in the CUDA library `libfairrank` (csrc/), reached through the C-ABI
declared in include/fairrank.h. `paper_2406_10262_gb300.fairrank` is the thin ctypes binding;
`paper_2406_10262_gb300.synth` generates seeded synthetic inputs. Importing the package loads
nothing: the binding loads the shared library on first use and raises if it is missing.
"""
__all__ = ["fairrank", "synth"]
