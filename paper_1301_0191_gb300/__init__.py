"""GB300 batched substructure engine for Adaptive-Multilevel BDDC
(Sousedik, Sistek, Mandel, arXiv:1301.0191).

The engine is the C-ABI library libamb.so (include/amb.h, sources in
csrc/, compiled by `build`); `binding` marshals arguments to it and
`autograd` wraps the adjoint gradient as a torch.autograd.Function.
"""
