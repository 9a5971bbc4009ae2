"""GB300-native periodic spin-orbital CCSD (arXiv:1911.00242).

The compute path is the C-ABI library libccsd_gb300.so (CUDA, sm_103a);
`binding` marshals arguments to it.  There is no CPU fallback: the library
must be built (`__graft_entry__.build()`) before use.
"""
