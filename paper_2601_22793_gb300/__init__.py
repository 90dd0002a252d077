"""GB300-native fast eikonal phase retrieval."""
