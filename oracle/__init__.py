"""FP64 CPU oracle of the APPGA hot path.  Test infrastructure only: the
tests, the package smoke check and the benchmark's CPU-baseline leg may
import it; the product path never does."""
