"""GB300-native fast-electron hybrid-PIC step (arXiv 2107.01723).

The CUDA library and its C-ABI live in `csrc/` and `include/hpic.h`; the
ctypes binding is `paper_2107_01723_gb300.hpic`.  Importing the package
loads nothing; the binding loads the library on first use and raises if it
is missing.
"""
