"""FP64 CPU oracle for the Kryging hot path.  Test infrastructure only: the test
suite, the package smoke check and the benchmark's CPU-baseline leg are its only
users; the product path never imports it."""
