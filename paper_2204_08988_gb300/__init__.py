"""GB300-native data-parallel hot path of the sub-cluster split/merge DPMM sampler
(arXiv 2204.08988).  The library loads lazily: importing the package (for example
for ``synth``) does not need a GPU."""
