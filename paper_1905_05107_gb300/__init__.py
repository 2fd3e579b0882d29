"""GB300-native iterative sampling-and-merging POD (arXiv 1905.05107).

The compute path lives in the CUDA shared library built from ``csrc/``;
``paper_1905_05107_gb300.pod`` is its thin ctypes binding.  Importing the
package loads nothing: the library is opened on first use.
"""
