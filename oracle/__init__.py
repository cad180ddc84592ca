"""Plain FP64 CPU oracle of the FSMP chain. Test infrastructure only: the CUDA product
path never imports this package."""
