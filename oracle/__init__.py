"""Plain FP64 CPU oracle for the phonon BTE hot path -- test infrastructure only."""
