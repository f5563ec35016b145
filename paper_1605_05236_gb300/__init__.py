"""GB300-native cuckoo hash tables with the kick-out policies and claim flags
of Kuszmaul, "Fast Concurrent Cuckoo Kick-out Eviction Schemes for
High-Density Tables" (arXiv:1605.05236).

The compute path is the CUDA library ``libck.so`` (C ABI in ``include/ck.h``);
``paper_1605_05236_gb300.ck`` is its thin Python binding.  Importing this
package loads nothing; the binding loads the library on first use and
raises if it is missing.
"""
