"""FP64 CPU oracle for the adaptive ray trace -- test infrastructure, not part of the library."""
