"""CPU FP64 oracle (test infrastructure only; see ``tdb_oracle``)."""
