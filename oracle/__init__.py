"""FP64 oracle of the inpainting hot path.  Test infrastructure only: tests, the smoke
check and the bench's CPU-baseline leg use it; the product path never imports it."""
